// sl_api.cu -- host side of libsl.so: the C ABI of include/sl.h.
//
// A context owns one device allocation holding two copies of the split
// coefficient store (ping-pong: every sweep reads one copy and writes the
// other), the per-shift-class tables, the mass-reduction partials and the
// field samples.  All device work goes to the context's stream; only calls
// that hand results to the host synchronise it.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sl_host.h"
#include "sl_nodal.h"

using namespace sl;
using namespace sl::host;

namespace {
thread_local std::string g_err;
// allocations left before the simulated failure (sl_debug_fail_alloc); 0: off
std::atomic<int64_t> g_fail_in{0};

bool simulated_failure()
{
    int64_t v = g_fail_in.load();
    while (v > 0) {
        if (g_fail_in.compare_exchange_weak(v, v - 1)) return v == 1;
    }
    return false;
}
}  // namespace

namespace sl {
namespace host {

sl_status fail_to(std::string* err, sl_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    *(err ? err : &g_err) = buf;
    return s;
}

sl_status fail(sl_ctx* c, sl_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_err = buf;
    return s;
}

cudaError_t dev_malloc(void** p, size_t bytes)
{
    if (simulated_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t pinned_malloc(void** p, size_t bytes)
{
    if (simulated_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

sl_status cuda_fail(sl_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, SL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}


size_t elem_size(int mode)
{
    switch (mode) {
    case M_FP64: return 8;
    case M_F32:
    case M_F32ALL:
    case M_SPLIT2:
    case M_SPLIT3: return 4;
    default: return 2;
    }
}

int64_t ipow(int64_t b, int e)
{
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

sl_status check_grid(const sl_grid* g, int degree, int storage, sl_ctx* c)
{
    if (!g) return fail(c, SL_EINVAL, "grid is NULL");
    if (g->ndim < 1 || g->ndim > SL_MAX_DIM)
        return fail(c, SL_EINVAL, "ndim must be in 1..%d (got %d)", SL_MAX_DIM, g->ndim);
    if (degree < 0 || degree > SL_MAX_DEGREE)
        return fail(c, SL_EINVAL, "degree must be in 0..%d (got %d)", SL_MAX_DEGREE, degree);
    if (storage < SL_FP64 || storage > SL_MIX_FP32_D3)
        return fail(c, SL_EINVAL, "unknown storage mode %d", storage);
    if (split_q(storage) > degree)
        return fail(c, SL_EINVAL, "# double = %d needs degree >= %d (got %d); degree + 1 is SL_FP64",
                    split_q(storage), split_q(storage), degree);
    double cells = 1.0;
    for (int m = 0; m < g->ndim; ++m) {
        if (g->n[m] < 1) return fail(c, SL_EINVAL, "n[%d] must be >= 1 (got %lld)", m, (long long)g->n[m]);
        if (!std::isfinite(g->lo[m]) || !std::isfinite(g->hi[m]) || !(g->hi[m] > g->lo[m]))
            return fail(c, SL_EINVAL, "dimension %d needs finite lo < hi", m);
        cells *= double(g->n[m]);
    }
    int used[SL_MAX_DIM] = {0};
    for (int m = 0; m < g->ndim; ++m) {
        const int p = g->pair[m];
        if (p == -1) continue;
        if (p < 0 || p >= g->ndim || p == m)
            return fail(c, SL_EINVAL, "pair[%d] = %d is not another dimension", m, p);
        if (g->pair[p] != -1) return fail(c, SL_EINVAL, "v-dimension %d is itself paired", p);
        if (used[p]++) return fail(c, SL_EINVAL, "v-dimension %d paired twice", p);
    }
    if (cells > double(0x7fffffff))
        return fail(c, SL_ENOTSUP, "grid has %.0f cells; this library indexes cells with 31 bits", cells);
    const int64_t nc = ipow(degree + 1, g->ndim);
    if ((storage == SL_MIX_BF16 || storage == SL_MIX_FP16) && nc > kMaxScaledCoef)
        return fail(c, SL_ENOTSUP, "scaled storage needs o^d <= %d (got %lld)", kMaxScaledCoef,
                    (long long)nc);
    return SL_OK;
}

void plane_counts(int ndim, int degree, int storage, int64_t* nlo, int64_t* nhi)
{
    const int64_t nc = ipow(degree + 1, ndim);
    const int q = split_q(storage);
    *nlo = q < 0 ? 1 : ipow(q, ndim);
    *nhi = nc - *nlo;
}

int64_t state_bytes_of(int64_t cells, int64_t nlo, int64_t nhi, int mode)
{
    int64_t b = cells * (8 * nlo + nhi * int64_t(elem_size(mode)));
    if (mode == M_BF16 || mode == M_FP16) b += cells * 4;
    return b;
}

double cell_width(const sl_grid& g, int m) { return (g.hi[m] - g.lo[m]) / double(g.n[m]); }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Guard bands of the context's allocation (sl_check_guards).
constexpr size_t kGuard = 256;
constexpr int kCanary = 0xA5;

bool is_scaled(const sl_ctx* c) { return c->mode == M_BF16 || c->mode == M_FP16; }
bool is_split(const sl_ctx* c) { return c->mode == M_SPLIT2 || c->mode == M_SPLIT3; }

void* hi_block(const sl_ctx* c, int parity)
{
    // the all-FP32 store's kernels address coefficient J at hi + (J-1)*pstride
    if (c->mode == M_F32ALL) return static_cast<float*>(c->planes[parity].hi) - c->pstride;
    return c->planes[parity].hi;
}

int64_t fibre_groups(const sl_ctx* c, int ft) { return is_scaled(c) ? 1 : (c->nfib + ft - 1) / ft; }

bool rec_lanes_ok(const sl_ctx* c) { return c->rec > 0 && c->K == 1 && (c->ndim == 5 || c->ndim == 6); }
bool rec_lanes(const sl_ctx* c, int ft) { return rec_lanes_ok(c) && ft == kRecLaneFt; }

// Chunk length of the strided walk: long enough to amortise the extra load at
// the start of a chunk, short enough to give a few waves of 2048 resident
// threads on every multiprocessor of the device, and no more than 65535 grid
// rows.
uint32_t chunk_for(const sl_ctx* c, int m, int ft, int lanes)
{
    const int64_t N = c->g.n[m];
    const int64_t lines = c->cells / N * lanes;
    const int64_t nfg = fibre_groups(c, ft);
    const int64_t want = int64_t(c->sm_count) * 2048 * 2;
    int64_t nchunk = (want + lines * nfg - 1) / (lines * nfg);
    if (nchunk < 1) nchunk = 1;
    int64_t chunk = (N + nchunk - 1) / nchunk;
    if (chunk < 4) chunk = 4;
    if (chunk > N) chunk = N;
    while (((N + chunk - 1) / chunk) * nfg > 65535) chunk *= 2;
    if (chunk > N) chunk = N;
    return uint32_t(chunk);
}

// Launch shapes compiled into the library.
bool unit_ft_ok(int ft) { return ft == 1 || ft == 2 || ft == 3 || ft == 4 || ft == 9; }
bool async_ok(int ft, int p) { return (p == 4 && ft >= 1 && ft <= 3) || (p == 8 && (ft == 1 || ft == 2)); }
bool strided_ok(int ft, int u)
{
    return (ft == 1 && (u == 1 || u == 2 || u == 4)) || (ft == 2 && (u == 1 || u == 2 || u == 4)) ||
           (ft == 3 && (u == 1 || u == 2));
}

// Cells per thread of the 16-byte vector form along dimension 0 (0 if the
// store or the extent does not allow it).
int unit_vec_width(const sl_ctx* c)
{
    if (is_scaled(c) || is_split(c)) return 0;
    const int v = int(16 / c->elem);
    return c->g.n[0] % v == 0 ? v : 0;
}

// Fibres per thread the scaled stores provide: the whole cell, or a split of
// its fibres over G cooperating threads (compiled splits only).
std::vector<int> scaled_fts(const sl_ctx* c)
{
    const int64_t nf = c->nfib;
    std::vector<int> v{int(nf)};
    if (rec_lanes_ok(c)) v.push_back(kRecLaneFt);
    if (c->rec) return v;   // otherwise a record is one thread's
    if (c->K == 1 && nf == 32) v.insert(v.end(), {16, 8, 4});
    if (c->K == 1 && nf == 16) v.insert(v.end(), {8, 4});
    if (c->K == 2 && nf == 27) v.insert(v.end(), {9, 3});
    if (c->K == 2 && nf == 9) v.push_back(3);
    if (c->K == 3 && nf == 16) v.push_back(4);
    return v;
}

// The smallest provided fibre count of at most 16 values per thread, else
// the whole cell.
int scaled_default_ft(const sl_ctx* c)
{
    int best = int(c->nfib);
    for (int f : scaled_fts(c))
        if (f * c->O <= 16 && (best * c->O > 16 || f > best)) best = f;
    return best;
}

// Default launch shape for a sweep along dimension m.
void default_tune(sl_ctx* c, int m)
{
    auto& t = c->tune[m];
    t.pipeline = 0;
    t.occ = 0;
    if (rec_lanes_ok(c) && c->ndim == 6) {
        // 128-byte records: lane groups (measured ahead of one thread per
        // cell, whose 16-byte pieces of 32 records per warp access keep the
        // L1 data pipe busy); every dimension is walked
        t.ft = kRecLaneFt;
        t.block = 128;
        t.unroll = m == 0 ? 2 : 1;
        t.chunk = chunk_for(c, m, 1, c->rec / 16);
        return;
    }
    // other records: one thread per cell (64-byte 5D records measured ahead of
    // lane groups)
    t.ft = c->rec ? int(c->nfib) : is_scaled(c) ? scaled_default_ft(c) : 1;
    if (is_split(c)) {   // one fibre per thread; no vector form
        t.block = m == 0 ? 256 : 128;
        t.unroll = m == 0 ? 1 : 2;
        t.chunk = m == 0 ? 0 : chunk_for(c, m, 1, 1);
        return;
    }
    if (m == 0) {
        t.block = c->rec ? 128 : 256;
        t.unroll = unit_vec_width(c) ? unit_vec_width(c) : 1;
        t.chunk = 0;
        return;
    }
    t.block = 128;
    t.unroll = is_scaled(c) ? 1 : 2;
    t.chunk = chunk_for(c, m, t.ft, 1);
}

SweepArgs make_args(sl_ctx* c, int dim, int shift_dim) { return make_args_parity(c, dim, shift_dim, c->cur); }

SweepArgs make_args_parity(sl_ctx* c, int dim, int shift_dim, int parity)
{
    SweepArgs a{};
    a.src = c->planes[parity];
    a.dst = c->planes[parity ^ 1];
    a.tab.sigma = c->d_sigma[dim];
    a.tab.alpha = c->d_alpha[dim];
    a.tab.ab64 = c->d_ab64[dim];
    a.tab.ab32 = c->d_ab32[dim];
    a.cells = uint32_t(c->cells);
    a.N = uint32_t(c->g.n[dim]);
    int64_t inner = 1;
    for (int q = 0; q < dim; ++q) inner *= c->g.n[q];
    a.inner = uint32_t(inner);
    a.lines = uint32_t(c->cells / c->g.n[dim]);
    a.pstride = c->pstride;
    a.fdN.set(a.N);
    a.fdInner.set(a.inner);
    if (shift_dim < 0) {
        a.cls_src = 0;
    } else {
        // The class is the coordinate along shift_dim.  For the strided
        // kernel a line is (outer, inner): shift_dim < dim lies in the inner
        // index, shift_dim > dim in the outer index.  The unit-stride kernel
        // (dim = 0) passes the line index as the outer index.
        int64_t div = 1;
        if (shift_dim < dim) {
            a.cls_src = 1;
            for (int q = 0; q < shift_dim; ++q) div *= c->g.n[q];
        } else {
            a.cls_src = 2;
            for (int q = dim + 1; q < shift_dim; ++q) div *= c->g.n[q];
        }
        a.fdCls.set(uint32_t(div));
        a.fdClsMod.set(uint32_t(c->g.n[shift_dim]));
    }
    a.ostride = int(ipow(c->O, dim));
    a.nfib = int(c->nfib);
    const auto& t = c->tune[dim];
    a.nfg = int(fibre_groups(c, t.ft));
    a.chunk = dim == 0 && !c->rec ? 0 : t.chunk;
    a.cmap = c->d_cmap;
    return a;
}

cudaEvent_t take_event(sl_ctx* c)
{
    if (!c->ev_free.empty()) {
        cudaEvent_t e = c->ev_free.back();
        c->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

cudaError_t launch_only(sl_ctx* c, int dim, int shift_dim)
{
    SweepLaunch L{};
    L.args = make_args(c, dim, shift_dim);
    L.K = c->K;
    L.mode = c->mode;
    L.unit = dim == 0;
    L.ft = c->tune[dim].ft;
    L.unroll = c->tune[dim].unroll;
    L.pipeline = dim == 0 ? 0 : c->tune[dim].pipeline;
    L.block = c->tune[dim].block;
    L.stream = c->st;
    L.dim = dim;
    L.ndim = c->ndim;
    L.rec = c->rec;
    L.occ = dim == 0 ? 0 : c->tune[dim].occ;
    if (c->wide) {   // FP64 arithmetic: one fibre per thread, its own walk chunk
        L.args.nfg = int(c->nfib);
        L.args.chunk = dim == 0 ? 0 : chunk_for(c, dim, 1, 1);
        return launch_sweep_wide(L);
    }
    if (is_scaled(c)) return launch_sweep_scaled(L);
    switch (c->mode) {
    case M_FP64: return launch_sweep_f64(L);
    case M_F32: return launch_sweep_f32(L);
    case M_F32ALL: return launch_sweep_f32all(L);
    default: return launch_sweep_split(L);
    }
}

// The nodal-in-velocity x-sweep along dim from the current copy, with the
// node table already built on the stream.
cudaError_t launch_nodal_only(sl_ctx* c, int dim)
{
    const int p = c->g.pair[dim];
    NodalArgs a{};
    a.src = c->planes[c->cur];
    a.dst = c->planes[c->cur ^ 1];
    a.tab.sigma = c->d_nsig;
    a.tab.alpha = c->d_nalpha;
    a.tab.ab64 = c->d_nab64;
    a.tab.ab32 = c->d_nab32;
    a.cells = uint32_t(c->cells);
    a.N = uint32_t(c->g.n[dim]);
    a.NV = uint32_t(c->g.n[p]);
    int64_t ix = 1, iv = 1;
    for (int q = 0; q < dim; ++q) ix *= c->g.n[q];
    for (int q = 0; q < p; ++q) iv *= c->g.n[q];
    a.inner_x = uint32_t(ix);
    a.fdInnerX.set(uint32_t(ix));
    a.fdNX.set(a.N);
    a.fdInnerV.set(uint32_t(iv));
    a.fdNV.set(a.NV);
    a.pstride = c->pstride;
    a.ostride = int(ipow(c->O, dim));
    a.vstride = int(ipow(c->O, p));
    a.ndim = c->ndim;
    a.xdim = dim;
    a.vdim = p;
    a.nfib2 = uint32_t(ipow(c->O, c->ndim - 2));
    a.off32 = double(c->pstride) * double(c->ncoef) < 2147483648.0 ? 1 : 0;
    double eta[kMaxO], w[kMaxO];
    nodal_setup(c->K, eta, w, &a);
    a.abar = c->d_nabar;
    a.na32 = c->d_nna32;
    return launch_sweep_nodal(c->K, c->mode, a, int(ipow(c->O, c->ndim - 2)), c->st);
}

// One sweep along dim using the shift table already built on the stream.
// Names of the NVTX ranges around each sweep launch (host-side markers that
// profilers show on the timeline; without an attached tool they cost a
// pointer test).
const char* const kSweepRange[2][SL_MAX_DIM] = {
    {"sl sweep dim 0", "sl sweep dim 1", "sl sweep dim 2", "sl sweep dim 3", "sl sweep dim 4", "sl sweep dim 5"},
    {"sl nodal sweep dim 0", "sl nodal sweep dim 1", "sl nodal sweep dim 2", "sl nodal sweep dim 3",
     "sl nodal sweep dim 4", "sl nodal sweep dim 5"}};

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

sl_status run_sweep(sl_ctx* c, int dim, int shift_dim, bool nodal = false)
{
    NvtxRange range(kSweepRange[nodal ? 1 : 0][dim]);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool prof = c->prof && !c->capturing;
    if (prof) {
        e0 = take_event(c);
        e1 = take_event(c);
        if (!e0 || !e1) return fail(c, SL_ECUDA, "cudaEventCreate failed");
        SL_CUDA(c, cudaEventRecord(e0, c->st));
    }
    cudaError_t e = nodal ? launch_nodal_only(c, dim) : launch_only(c, dim, shift_dim);
    if (e != cudaSuccess) return cuda_fail(c, e, "sweep kernel launch");
    if (prof) {
        SL_CUDA(c, cudaEventRecord(e1, c->st));
        c->ev_used.emplace_back(e0, e1);
        c->ev_dim.push_back(dim);
        c->prof_launches++;
    }
    c->cur ^= 1;
    return SL_OK;
}

// Node table of the x-sweep along dim over time tau: class j * o + q has
// the velocity of node q of v-cell j.
sl_status nodal_table(sl_ctx* c, int dim, double tau)
{
    const int p = c->g.pair[dim];
    ShiftSource src{};
    src.kind = 2;
    src.data = static_cast<const double*>(c->d_nodal) + c->nodal_vel_off[dim];
    src.tau = tau;
    src.h = cell_width(c->g, dim);
    cudaError_t e = launch_ab_build(c->K, int(c->g.n[p] * c->O), uint32_t(c->g.n[dim]), src, c->poly, c->d_nsig,
                                    c->d_nalpha, c->d_nab64, c->d_nab32, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "node table launch");
    if (c->mode == M_F32) {   // alpha_bar per v-cell for the mean's fibre
        NodalArgs tmp{};
        double eta[kMaxO], w[kMaxO];
        nodal_setup(c->K, eta, w, &tmp);
        e = launch_nodal_abar(c->d_nalpha, int(c->g.n[p]), c->O, tmp.wmean, tmp.wmean32, c->d_nabar, c->d_nna32,
                              c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "node table launch");
    }
    return SL_OK;
}

// The shift table of dimension dim (its own slot) on stream st.
sl_status build_table_on(sl_ctx* c, int dim, int nclass, const ShiftSource& src, cudaStream_t st)
{
    if (nclass < 1 || nclass > c->ncls[dim])
        return fail(c, SL_EINVAL, "%d shift classes for dimension %d (at most %d)", nclass, dim, c->ncls[dim]);
    cudaError_t e = launch_ab_build(c->K, nclass, uint32_t(c->g.n[dim]), src, c->poly, c->d_sigma[dim],
                                    c->d_alpha[dim], c->d_ab64[dim], c->d_ab32[dim], st);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_build launch");
    return SL_OK;
}

sl_status build_table(sl_ctx* c, int dim, int nclass, const ShiftSource& src)
{
    return build_table_on(c, dim, nclass, src, c->st);
}

// The sweeps of one split step: (dim, tau factor).
std::vector<SubStep> plan_of(const sl_ctx* c, sl_splitting sp)
{
    std::vector<int> xd, vd;
    for (int m = 0; m < c->ndim; ++m)
        if (c->g.pair[m] >= 0) {
            xd.push_back(m);
            vd.push_back(c->g.pair[m]);
        }
    std::vector<SubStep> p;
    if (sp == SL_STRANG) {
        for (int m : xd) p.push_back({m, 0.5});
        for (int v : vd) p.push_back({v, 1.0});
        for (int m : xd) p.push_back({m, 0.5});
    } else {
        for (int m : xd) p.push_back({m, 1.0});
        for (int v : vd) p.push_back({v, 1.0});
    }
    return p;
}

// Offset of the field of x-dimension m inside d_fields.
int64_t field_offset(const sl_ctx* c, int xdim)
{
    int64_t off = 0;
    for (int m = 0; m < xdim; ++m)
        if (c->g.pair[m] >= 0) off += c->g.n[m];
    return off;
}

// Field of the current state at the x-cell centres into E (and the field
// energy into *energy) on the context's stream.
cudaError_t vp_field(sl_ctx* c, double* E, double* energy)
{
    const int x = c->vp_x, v = c->vp_v;
    const uint32_t nx = uint32_t(c->g.n[x]), nv = uint32_t(c->g.n[v]);
    const uint32_t sx = x == 0 ? 1u : uint32_t(c->g.n[0]);
    const uint32_t sv = v == 0 ? 1u : uint32_t(c->g.n[0]);
    return launch_vp_field(c->planes[c->cur].mean, nx, nv, sx, sv, cell_width(c->g, x), cell_width(c->g, v),
                           c->d_vp, E, energy, c->st);
}

// Shift source of a split substep's sweep along dim over tau (not the nodal
// x-sweep): x-dimensions take the centre velocity of their v-dimension, the
// v-dimensions the field on the x-grid (the self-consistent field first
// computed from the current state when `field` is set).
sl_status substep_source(sl_ctx* c, int dim, double tau, bool field, ShiftSource* src, int* shift_dim,
                         int* nclass)
{
    *src = ShiftSource{};
    if (c->g.pair[dim] >= 0) {
        const int p = c->g.pair[dim];
        src->kind = 1;
        src->lo = c->g.lo[p];
        src->hv = cell_width(c->g, p);
        src->tau = tau;
        src->h = cell_width(c->g, dim);
        *shift_dim = p;
        *nclass = int(c->g.n[p]);
        return SL_OK;
    }
    int xm = -1;
    for (int m = 0; m < c->ndim; ++m)
        if (c->g.pair[m] == dim) xm = m;
    if (field && c->poisson) {   // the field of the current state
        cudaError_t e = vp_field(c, c->d_fields + field_offset(c, xm), nullptr);
        if (e != cudaSuccess) return cuda_fail(c, e, "self-consistent field");
    }
    src->kind = 2;
    src->data = c->d_fields + field_offset(c, xm);
    src->tau = tau;
    src->h = cell_width(c->g, dim);
    *shift_dim = xm;
    *nclass = int(c->g.n[xm]);
    return SL_OK;
}

// The split steps.  A shift table depends on its dimension, tau and the
// fields, not on the state, so each dimension's table is built once per
// step into its own slot (Strang's two x half-steps share theirs): the
// x-dimensions' on the context's stream before the step's first sweep, the
// v-dimensions' on the side stream while the x-sweeps run, joined back before
// the first v-sweep.  With the self-consistent field a v-table needs the
// field of the state after the x-sweeps, so it is built right before its
// sweep, after the field.
sl_status enqueue_steps(sl_ctx* c, sl_splitting sp, double dt, int nsteps)
{
    const std::vector<SubStep> plan = plan_of(c, sp);
    bool ahead = true;
    for (const SubStep& a : plan)
        for (const SubStep& b : plan)
            if (a.dim == b.dim && a.frac != b.frac) ahead = false;
    for (int s = 0; s < nsteps; ++s) {
        bool built[SL_MAX_DIM] = {false};
        bool joined = true;
        if (ahead) {
            bool any_v = false;
            for (const SubStep& ss : plan) {
                const bool x = c->g.pair[ss.dim] >= 0;
                if (x && c->nodal) continue;   // node tables: before each nodal sweep
                if (!x) {
                    any_v = any_v || !c->poisson;
                    continue;
                }
                if (built[ss.dim]) continue;
                ShiftSource src;
                int sd, nclass;
                sl_status r = substep_source(c, ss.dim, ss.frac * dt, false, &src, &sd, &nclass);
                if (r == SL_OK) r = build_table(c, ss.dim, nclass, src);
                if (r != SL_OK) return r;
                built[ss.dim] = true;
            }
            if (any_v) {
                SL_CUDA(c, cudaEventRecord(c->ev_fork, c->st));
                SL_CUDA(c, cudaStreamWaitEvent(c->st_tab, c->ev_fork, 0));
                for (const SubStep& ss : plan) {
                    if (c->g.pair[ss.dim] >= 0 || built[ss.dim] || c->poisson) continue;
                    ShiftSource src;
                    int sd, nclass;
                    sl_status r = substep_source(c, ss.dim, ss.frac * dt, false, &src, &sd, &nclass);
                    if (r == SL_OK) r = build_table_on(c, ss.dim, nclass, src, c->st_tab);
                    if (r != SL_OK) return r;
                    built[ss.dim] = true;
                }
                SL_CUDA(c, cudaEventRecord(c->ev_join, c->st_tab));
                joined = false;
            }
        }
        for (const SubStep& ss : plan) {
            const double tau = ss.frac * dt;
            if (c->g.pair[ss.dim] >= 0 && c->nodal) {
                // x-sweep with the velocity at the Gauss nodes of every v-cell
                sl_status r = nodal_table(c, ss.dim, tau);
                if (r == SL_OK) r = run_sweep(c, ss.dim, -1, true);
                if (r != SL_OK) return r;
                continue;
            }
            ShiftSource src;
            int shift_dim, nclass;
            sl_status r = substep_source(c, ss.dim, tau, !built[ss.dim], &src, &shift_dim, &nclass);
            if (r != SL_OK) return r;
            if (!built[ss.dim]) {
                r = build_table(c, ss.dim, nclass, src);
                if (r != SL_OK) return r;
            } else if (!joined && c->g.pair[ss.dim] < 0) {
                SL_CUDA(c, cudaStreamWaitEvent(c->st, c->ev_join, 0));
                joined = true;
            }
            r = run_sweep(c, ss.dim, shift_dim);
            if (r != SL_OK) return r;
        }
        if (!joined) SL_CUDA(c, cudaStreamWaitEvent(c->st, c->ev_join, 0));
    }
    return SL_OK;
}

sl_status ensure_stage(sl_ctx* c)
{
    if (c->d_stage) return SL_OK;
    const int64_t bytes_target = int64_t(64) << 20;
    int64_t n = bytes_target / (c->ncoef * 8);
    if (n < 1) n = 1;
    if (n > c->cells) n = c->cells;
    void* p = nullptr;
    cudaError_t e = dev_malloc(&p, size_t(n) * c->ncoef * 8);
    if (e != cudaSuccess) return fail(c, SL_ENOMEM, "staging allocation: %s", cudaGetErrorString(e));
    c->d_stage = static_cast<double*>(p);
    c->stage_cells = n;
    return SL_OK;
}

CodecArgs codec_of(const sl_ctx* c)
{
    CodecArgs a{};
    a.p = c->planes[c->cur];
    a.pstride = c->pstride;
    a.ncoef = int(c->ncoef);
    a.mode = c->mode;
    a.rec = c->rec;
    a.cmap = c->d_cmap;
    if (is_split_family(c->mode)) a.p.hi = hi_block(c, c->cur);
    return a;
}

void drop_graph(sl_ctx* c)
{
    for (auto& g : c->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    c->graph_start = -1;
}

int natural_shift_dim(const sl_ctx* c, int m)
{
    if (c->g.pair[m] >= 0) return c->g.pair[m];
    for (int q = 0; q < c->ndim; ++q)
        if (c->g.pair[q] == m) return q;
    return -1;
}

}  // namespace host
}  // namespace sl

// ======================================================================
// ABI
// ======================================================================

namespace {

// Capture `sweeps` sweeps issued by `enqueue` into one graph, or into two when
// `sweeps` is odd (the graph for each copy of the ping-pong state it may start
// from).
template <typename F>
sl_status capture_graphs(sl_ctx* c, int sweeps, F enqueue)
{
    if (!c->st) return fail(c, SL_EINVAL, "graph capture needs a non-default stream");
    drop_graph(c);
    const int start = c->cur;
    const int flip = sweeps & 1;
    const int ngraphs = flip ? 2 : 1;
    for (int gi = 0; gi < ngraphs; ++gi) {
        c->cur = start ^ gi;
        cudaGraph_t graph = nullptr;
        SL_CUDA(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        c->capturing = true;
        sl_status s = enqueue();
        c->capturing = false;
        cudaError_t e = cudaStreamEndCapture(c->st, &graph);
        if (s != SL_OK) {
            if (graph) cudaGraphDestroy(graph);
            c->cur = start;
            drop_graph(c);
            return s;
        }
        if (e != cudaSuccess) {
            c->cur = start;
            drop_graph(c);
            return cuda_fail(c, e, "cudaStreamEndCapture");
        }
        e = cudaGraphInstantiate(&c->gexec[gi], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->cur = start;
            drop_graph(c);
            return cuda_fail(c, e, "cudaGraphInstantiate");
        }
    }
    c->cur = start;
    c->graph_start = start;
    c->graph_flip = flip;
    return SL_OK;
}

}  // namespace

extern "C" {

const char* sl_last_error(const sl_ctx* ctx)
{
    if (ctx) return ctx->err.c_str();
    return g_err.c_str();
}

sl_status sl_state_bytes(const sl_grid* grid, int degree, sl_storage storage, int64_t* bytes)
{
    sl_status s = check_grid(grid, degree, storage, nullptr);
    if (s != SL_OK) return s;
    if (!bytes) return fail(nullptr, SL_EINVAL, "bytes is NULL");
    int64_t cells = 1;
    for (int m = 0; m < grid->ndim; ++m) cells *= grid->n[m];
    int64_t nlo, nhi;
    plane_counts(grid->ndim, degree, storage, &nlo, &nhi);
    *bytes = state_bytes_of(cells, nlo, nhi, storage);
    return SL_OK;
}

sl_status sl_ab_host(int degree, double alpha, double* A, double* B)
{
    if (degree < 0 || degree > SL_MAX_DEGREE) return fail(nullptr, SL_EINVAL, "degree out of range");
    if (!(alpha >= 0.0) || !(alpha < 1.0)) return fail(nullptr, SL_EINVAL, "alpha must be in [0,1)");
    if (!A || !B) return fail(nullptr, SL_EINVAL, "NULL output");
    PolyTab t;
    build_poly_table(degree, &t);
    const int O = degree + 1, deg = 2 * degree + 1;
    const double x = alpha - 0.5;
    for (int j = 0; j < O; ++j)
        for (int l = 0; l < O; ++l) {
            double va, vb;
            if (alpha == 0.0) {
                va = j == l ? 1.0 : 0.0;
                vb = 0.0;
            } else {
                va = t.a[j][l][deg];
                vb = t.b[j][l][deg];
                for (int p = deg - 1; p >= 0; --p) {
                    va = std::fma(va, x, t.a[j][l][p]);
                    vb = std::fma(vb, x, t.b[j][l][p]);
                }
            }
            A[j * O + l] = va;
            B[j * O + l] = vb;
        }
    return SL_OK;
}

// One copy of the state: bytes of the mean plane, the higher coefficients
// (planes or cell records) and the scale plane (0 for the unscaled stores).
static void copy_bytes(int64_t cells, int64_t nlo, int64_t nhi, int rec, int elem, bool scaled, int64_t pstride,
                       size_t* mean, size_t* hi, size_t* scale)
{
    *mean = size_t(pstride) * size_t(nlo) * 8;
    *hi = rec ? size_t(cells) * size_t(rec) * size_t(elem) : size_t(pstride) * size_t(nhi) * size_t(elem);
    *scale = scaled ? size_t(pstride) * 4 : 0;
}

// Coefficient map of the stores of # double = q (sl::Planes): FP64 plane
// -1 - e or FP32 plane e for every coefficient J, each block in increasing J.
// The all-FP32 store (q = 0) maps J to FP32 plane J.
static std::vector<int32_t> coefficient_map(int ndim, int O, int q)
{
    const int64_t nc = ipow(O, ndim);
    std::vector<int32_t> map(size_t(nc), 0);
    int32_t nlo = 0, nhi = 0;
    for (int64_t J = 0; J < nc; ++J) {
        bool lo = true;
        int64_t r = J;
        for (int m = 0; m < ndim; ++m) {
            lo = lo && (r % O) < q;
            r /= O;
        }
        map[size_t(J)] = lo ? -1 - nlo++ : nhi++;
    }
    return map;
}

static int record_slots_of(const sl_grid* grid, int degree, sl_storage storage, int64_t ncoef)
{
    // cell records for the scaled shapes that fill them (at most one padding
    // slot besides slot 0): 6D and 5D with k = 1, 3D with k = 3
    if ((storage == SL_MIX_BF16 || storage == SL_MIX_FP16) &&
        ((degree == 1 && (grid->ndim == 6 || grid->ndim == 5)) || (degree == 3 && grid->ndim == 3)))
        return int((ncoef + 7) / 8 * 8);
    return 0;
}

// planes == nullptr: the context allocates both copies of the state;
// otherwise planes = {mean0, hi0, scale0, mean1, hi1, scale1}, caller-owned.
static sl_status create_ctx(const sl_grid* grid, int degree, sl_storage storage, void* cuda_stream,
                            void* const* planes, sl_ctx** out)
{
    if (!out) return fail(nullptr, SL_EINVAL, "out is NULL");
    *out = nullptr;
    sl_status s = check_grid(grid, degree, storage, nullptr);
    if (s != SL_OK) return s;
    const bool scaled = storage == SL_MIX_BF16 || storage == SL_MIX_FP16;
    if (planes)
        for (int q = 0; q < 6; ++q) {
            const bool need = (q % 3 == 0 && storage != SL_FP32) || q % 3 == 1 || scaled;
            if (need && !planes[q]) return fail(nullptr, SL_EINVAL, "plane pointer %d is NULL", q);
            if (planes[q] && reinterpret_cast<uintptr_t>(planes[q]) % 256 != 0)
                return fail(nullptr, SL_EINVAL, "plane pointer %d is not 256-byte aligned", q);
        }

    sl_ctx* c = new (std::nothrow) sl_ctx();
    if (!c) return fail(nullptr, SL_ENOMEM, "host allocation failed");
    c->g = *grid;
    for (int m = c->g.ndim; m < SL_MAX_DIM; ++m) {
        c->g.n[m] = 1;
        c->g.pair[m] = -1;
    }
    c->K = degree;
    c->O = degree + 1;
    c->ndim = grid->ndim;
    c->mode = Mode(storage);
    c->st = static_cast<cudaStream_t>(cuda_stream);
    c->cells = 1;
    for (int m = 0; m < c->ndim; ++m) c->cells *= grid->n[m];
    c->ncoef = ipow(c->O, c->ndim);
    c->nfib = ipow(c->O, c->ndim - 1);
    c->pstride = int64_t(align_up(size_t(c->cells), 64));
    c->elem = elem_size(storage);
    c->rec = record_slots_of(grid, degree, storage, c->ncoef);
    plane_counts(c->ndim, degree, storage, &c->nlo, &c->nhi);
    c->state_bytes = state_bytes_of(c->cells, c->nlo, c->nhi, storage);
    c->external = planes != nullptr;
    for (int m = 0; m < c->ndim; ++m) {
        c->ncls[m] = 1;
        for (int q = 0; q < c->ndim; ++q)
            if (q != m) c->ncls[m] = std::max<int>(c->ncls[m], int(c->g.n[q]));
        c->maxcls = std::max(c->maxcls, c->ncls[m]);
    }
    build_poly_table(degree, &c->poly);
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || c->sm_count < 1) {
            delete c;
            return fail(nullptr, SL_ECUDA, "querying the device's multiprocessor count: %s", cudaGetErrorString(e));
        }
    }
    for (int m = 0; m < c->ndim; ++m) default_tune(c, m);

    // layout of the single allocation (the state only when the context owns
    // it): every array 256-B aligned and followed by a guard band of at least
    // kGuard bytes filled with kCanary (sl_check_guards)
    const size_t A = 256;
    size_t off = 0;
    auto place = [&](size_t bytes) {
        const size_t at = off;
        const size_t end = at + bytes;
        off = align_up(end + kGuard, A);
        c->bands.push_back({end, 0, off - end, 1});
        return at;
    };
    size_t o_state[2][3] = {{0, 0, 0}, {0, 0, 0}};
    size_t b_mean, b_hi, b_scale;
    copy_bytes(c->cells, c->nlo, c->nhi, c->rec, c->elem, scaled, c->pstride, &b_mean, &b_hi, &b_scale);
    if (!planes)
        for (int b = 0; b < 2; ++b) {
            o_state[b][0] = place(b_mean);
            o_state[b][1] = place(b_hi);
            o_state[b][2] = place(b_scale);
            // the planes' padding past the last cell
            const size_t pad = size_t(c->pstride - c->cells);
            if (pad > 0) {
                if (c->nlo > 0) c->bands.push_back({o_state[b][0] + size_t(c->cells) * 8, size_t(c->pstride) * 8, pad * 8,
                                                    size_t(c->nlo)});
                if (!c->rec && c->nhi > 0)
                    c->bands.push_back({o_state[b][1] + size_t(c->cells) * c->elem, size_t(c->pstride) * c->elem,
                                        pad * c->elem, size_t(c->nhi)});
                if (scaled) c->bands.push_back({o_state[b][2] + size_t(c->cells) * 4, 0, pad * 4, 1});
            }
        }
    size_t o_sigma[SL_MAX_DIM], o_alpha[SL_MAX_DIM], o_ab64[SL_MAX_DIM], o_ab32[SL_MAX_DIM];
    for (int m = 0; m < c->ndim; ++m) {
        const size_t n = size_t(c->ncls[m]);
        o_sigma[m] = place(n * 4);
        o_alpha[m] = place(n * 8);
        o_ab64[m] = place(n * ab_stride64(c->O) * 8);
        o_ab32[m] = place(n * ab_stride32(c->O) * 4);
    }
    const size_t o_shifts = place(size_t(c->maxcls) * 8);
    int64_t nf = 0;
    for (int m = 0; m < c->ndim; ++m)
        if (c->g.pair[m] >= 0) nf += c->g.n[m];
    c->nfields = nf;
    const size_t o_fields = place(size_t(std::max<int64_t>(nf, 1)) * 8);
    c->mass_nblk = mass_blocks(uint32_t(c->cells));
    const size_t o_part = place(size_t(c->mass_nblk) * 8);
    const size_t o_mass = place(8);
    const bool mapped = is_split_family(c->mode);
    const size_t o_cmap = mapped ? place(size_t(c->ncoef) * 4) : 0;
    c->mem_bytes = off;

    cudaError_t e = dev_malloc(&c->mem, c->mem_bytes);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, SL_ENOMEM, "cudaMalloc(%zu bytes): %s", off, cudaGetErrorString(e));
    }
    char* base = static_cast<char*>(c->mem);
    for (int b = 0; b < 2; ++b) {
        if (planes) {
            c->planes[b].mean = static_cast<double*>(planes[3 * b]);
            c->planes[b].hi = planes[3 * b + 1];
            c->planes[b].scale = scaled ? static_cast<float*>(planes[3 * b + 2]) : nullptr;
        } else {
            c->planes[b].mean = reinterpret_cast<double*>(base + o_state[b][0]);
            c->planes[b].hi = base + o_state[b][1];
            c->planes[b].scale = scaled ? reinterpret_cast<float*>(base + o_state[b][2]) : nullptr;
        }
        if (c->mode == M_F32ALL) {   // see sl::Planes
            c->planes[b].mean = nullptr;
            c->planes[b].hi = static_cast<float*>(c->planes[b].hi) + c->pstride;
        }
    }
    if (mapped) c->d_cmap = reinterpret_cast<int32_t*>(base + o_cmap);
    for (int m = 0; m < c->ndim; ++m) {
        c->d_sigma[m] = reinterpret_cast<int32_t*>(base + o_sigma[m]);
        c->d_alpha[m] = reinterpret_cast<double*>(base + o_alpha[m]);
        c->d_ab64[m] = reinterpret_cast<double*>(base + o_ab64[m]);
        c->d_ab32[m] = reinterpret_cast<float*>(base + o_ab32[m]);
    }
    c->d_shifts = reinterpret_cast<double*>(base + o_shifts);
    c->d_fields = reinterpret_cast<double*>(base + o_fields);
    c->d_partials = reinterpret_cast<double*>(base + o_part);
    c->d_mass = reinterpret_cast<double*>(base + o_mass);
    e = pinned_malloc(reinterpret_cast<void**>(&c->h_mass), 8);
    if (e != cudaSuccess) {
        cudaFree(c->mem);
        delete c;
        return fail(nullptr, SL_ENOMEM, "cudaMallocHost: %s", cudaGetErrorString(e));
    }
    // an owned state starts at zero (the scale plane at zero decodes to zero
    // too); a caller's planes keep their contents
    e = cudaMemsetAsync(c->mem, 0, c->mem_bytes, c->st);
    for (const auto& bd : c->bands) {
        if (e != cudaSuccess) break;
        char* at = static_cast<char*>(c->mem) + bd.off;
        e = bd.height == 1 ? cudaMemsetAsync(at, kCanary, bd.width, c->st)
                           : cudaMemset2DAsync(at, bd.pitch, kCanary, bd.width, bd.height, c->st);
    }
    std::vector<int32_t> cmap;
    if (mapped && e == cudaSuccess) {
        cmap = coefficient_map(c->ndim, c->O, split_q(c->mode));
        e = cudaMemcpyAsync(c->d_cmap, cmap.data(), cmap.size() * 4, cudaMemcpyHostToDevice, c->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->st_tab, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->st_tab) cudaStreamDestroy(c->st_tab);
        cudaFreeHost(c->h_mass);
        cudaFree(c->mem);
        delete c;
        return fail(nullptr, SL_ECUDA, "initialising the state: %s", cudaGetErrorString(e));
    }
    *out = c;
    return SL_OK;
}

sl_status sl_create(const sl_grid* grid, int degree, sl_storage storage, void* cuda_stream, sl_ctx** out)
{
    return create_ctx(grid, degree, storage, cuda_stream, nullptr, out);
}

sl_status sl_create_external(const sl_grid* grid, int degree, sl_storage storage, void* cuda_stream,
                             void* const* planes, sl_ctx** out)
{
    if (!planes) return fail(nullptr, SL_EINVAL, "planes is NULL");
    return create_ctx(grid, degree, storage, cuda_stream, planes, out);
}

sl_status sl_plane_layout(const sl_grid* grid, int degree, sl_storage storage, sl_layout* out)
{
    if (!out) return fail(nullptr, SL_EINVAL, "out is NULL");
    sl_status s = check_grid(grid, degree, storage, nullptr);
    if (s != SL_OK) return s;
    int64_t cells = 1;
    for (int m = 0; m < grid->ndim; ++m) cells *= grid->n[m];
    const int64_t ncoef = ipow(degree + 1, grid->ndim);
    const int64_t pstride = int64_t(align_up(size_t(cells), 64));
    const int rec = record_slots_of(grid, degree, storage, ncoef);
    int64_t nlo, nhi;
    plane_counts(grid->ndim, degree, storage, &nlo, &nhi);
    size_t bm, bh, bs;
    copy_bytes(cells, nlo, nhi, rec, elem_size(storage), storage == SL_MIX_BF16 || storage == SL_MIX_FP16, pstride,
               &bm, &bh, &bs);
    out->plane_stride = pstride;
    out->record_slots = rec;
    out->reserved = 0;
    out->mean_bytes = int64_t(bm);
    out->hi_bytes = int64_t(bh);
    out->scale_bytes = int64_t(bs);
    return SL_OK;
}

sl_status sl_debug_fail_alloc(int64_t n)
{
    if (n < 0) return fail(nullptr, SL_EINVAL, "n must be >= 0");
    g_fail_in.store(n);
    return SL_OK;
}

sl_status sl_check_guards(sl_ctx* c, int64_t* corrupted)
{
    if (!c || !corrupted) return fail(c, SL_EINVAL, "NULL argument");
    if (c->capturing) return fail(c, SL_EINVAL, "cannot check the guards during a capture");
    *corrupted = 0;
    std::vector<unsigned char> buf;
    for (const auto& bd : c->bands) {
        if (bd.width == 0 || bd.height == 0) continue;
        buf.resize(bd.width * bd.height);
        const char* at = static_cast<const char*>(c->mem) + bd.off;
        if (bd.height == 1)
            SL_CUDA(c, cudaMemcpyAsync(buf.data(), at, bd.width, cudaMemcpyDeviceToHost, c->st));
        else
            SL_CUDA(c, cudaMemcpy2DAsync(buf.data(), bd.width, at, bd.pitch, bd.width, bd.height,
                                         cudaMemcpyDeviceToHost, c->st));
        SL_CUDA(c, cudaStreamSynchronize(c->st));
        for (unsigned char x : buf) *corrupted += x != kCanary;
    }
    return SL_OK;
}

sl_status sl_debug_corrupt_guard(sl_ctx* c)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (c->bands.empty()) return fail(c, SL_EINVAL, "no guard band");
    const unsigned char zero = 0;
    SL_CUDA(c, cudaMemcpyAsync(static_cast<char*>(c->mem) + c->bands.front().off, &zero, 1, cudaMemcpyHostToDevice,
                               c->st));
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    return SL_OK;
}

void sl_destroy(sl_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    drop_graph(c);
    for (auto& pr : c->ev_used) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto e : c->ev_free) cudaEventDestroy(e);
    if (c->d_stage) cudaFree(c->d_stage);
    if (c->d_proj) cudaFree(c->d_proj);
    if (c->d_vp) cudaFree(c->d_vp);
    if (c->d_nodal) cudaFree(c->d_nodal);
    if (c->d_gshifts) cudaFree(c->d_gshifts);
    if (c->h_mass) cudaFreeHost(c->h_mass);
    if (c->mem) cudaFree(c->mem);   // a caller's planes (sl_create_external) are not freed
    if (c->st_tab) {
        cudaStreamSynchronize(c->st_tab);
        cudaStreamDestroy(c->st_tab);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
}

sl_status sl_get_info(const sl_ctx* c, sl_info* out)
{
    if (!c || !out) return fail(nullptr, SL_EINVAL, "NULL argument");
    out->cells = c->cells;
    out->ncoef = c->ncoef;
    out->dof = c->cells * c->ncoef;
    out->plane_stride = c->pstride;
    out->state_bytes = c->state_bytes;
    out->alloc_bytes = int64_t(c->mem_bytes) + (c->d_stage ? c->stage_cells * c->ncoef * 8 : 0) +
                       int64_t(c->proj_bytes);
    out->degree = c->K;
    out->storage = c->mode;
    out->record_slots = c->rec;
    return SL_OK;
}

sl_status sl_set_coeffs(sl_ctx* c, const double* host)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (!host) return fail(c, SL_EINVAL, "host array is NULL");
    const int64_t n = c->cells * c->ncoef;
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(host[i])) return fail(c, SL_ENAN, "non-finite coefficient at index %lld", (long long)i);
    sl_status s = ensure_stage(c);
    if (s != SL_OK) return s;
    const CodecArgs ca = codec_of(c);
    for (int64_t first = 0; first < c->cells; first += c->stage_cells) {
        const int64_t cnt = std::min(c->stage_cells, c->cells - first);
        SL_CUDA(c, cudaMemcpyAsync(c->d_stage, host + first * c->ncoef, size_t(cnt) * c->ncoef * 8,
                                   cudaMemcpyHostToDevice, c->st));
        SL_CUDA(c, launch_encode(ca, c->d_stage, uint32_t(first), uint32_t(cnt), c->st));
    }
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    return SL_OK;
}

sl_status sl_get_coeffs(sl_ctx* c, double* host)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (!host) return fail(c, SL_EINVAL, "host array is NULL");
    sl_status s = ensure_stage(c);
    if (s != SL_OK) return s;
    const CodecArgs ca = codec_of(c);
    for (int64_t first = 0; first < c->cells; first += c->stage_cells) {
        const int64_t cnt = std::min(c->stage_cells, c->cells - first);
        SL_CUDA(c, launch_decode(ca, c->d_stage, uint32_t(first), uint32_t(cnt), c->st));
        SL_CUDA(c, cudaMemcpyAsync(host + first * c->ncoef, c->d_stage, size_t(cnt) * c->ncoef * 8,
                                   cudaMemcpyDeviceToHost, c->st));
        SL_CUDA(c, cudaStreamSynchronize(c->st));
    }
    return SL_OK;
}

sl_status sl_get_cells(sl_ctx* c, const int64_t* cells, int64_t ncells, double* host)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (ncells < 0 || (ncells > 0 && (!cells || !host))) return fail(c, SL_EINVAL, "bad cell list");
    if (ncells == 0) return SL_OK;
    for (int64_t i = 0; i < ncells; ++i)
        if (cells[i] < 0 || cells[i] >= c->cells)
            return fail(c, SL_EINVAL, "cell index %lld out of range", (long long)cells[i]);
    sl_status s = ensure_stage(c);
    if (s != SL_OK) return s;
    // stage layout: [idx block of int64][values]
    const CodecArgs ca = codec_of(c);
    const int64_t per = std::max<int64_t>(1, (c->stage_cells * c->ncoef * 8) / (8 + c->ncoef * 8));
    for (int64_t first = 0; first < ncells; first += per) {
        const int64_t cnt = std::min(per, ncells - first);
        int64_t* d_idx = reinterpret_cast<int64_t*>(c->d_stage);
        double* d_val = c->d_stage + cnt;
        SL_CUDA(c, cudaMemcpyAsync(d_idx, cells + first, size_t(cnt) * 8, cudaMemcpyHostToDevice, c->st));
        SL_CUDA(c, launch_gather(ca, d_idx, uint32_t(cnt), d_val, c->st));
        SL_CUDA(c, cudaMemcpyAsync(host + first * c->ncoef, d_val, size_t(cnt) * c->ncoef * 8,
                                   cudaMemcpyDeviceToHost, c->st));
        SL_CUDA(c, cudaStreamSynchronize(c->st));
    }
    return SL_OK;
}

static sl_status planes_args(sl_ctx* c, const void* mean, const void* hi, const void* scale)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    const bool scaled = c->mode == M_BF16 || c->mode == M_FP16;
    if ((c->nlo > 0 && !mean) || (c->nhi > 0 && !hi)) return fail(c, SL_EINVAL, "NULL plane");
    if (scaled && !scale) return fail(c, SL_EINVAL, "scaled store needs the scale plane");
    if (c->capturing) return fail(c, SL_EINVAL, "plane copies cannot be captured");
    return SL_OK;
}

sl_status sl_set_planes(sl_ctx* c, const double* mean, const void* hi, const float* scale)
{
    sl_status s = planes_args(c, mean, hi, scale);
    if (s != SL_OK) return s;
    const Planes& p = c->planes[c->cur];
    void* hb = hi_block(c, c->cur);
    if (c->nlo > 0)
        SL_CUDA(c, cudaMemcpy2DAsync(p.mean, size_t(c->pstride) * 8, mean, size_t(c->cells) * 8,
                                     size_t(c->cells) * 8, size_t(c->nlo), cudaMemcpyHostToDevice, c->st));
    if (c->rec)
        SL_CUDA(c, cudaMemcpyAsync(hb, hi, size_t(c->cells) * c->rec * c->elem, cudaMemcpyHostToDevice,
                                   c->st));
    else if (c->nhi > 0)
        SL_CUDA(c, cudaMemcpy2DAsync(hb, size_t(c->pstride) * c->elem, hi, size_t(c->cells) * c->elem,
                                     size_t(c->cells) * c->elem, size_t(c->nhi),
                                     cudaMemcpyHostToDevice, c->st));
    if (p.scale)
        SL_CUDA(c, cudaMemcpyAsync(p.scale, scale, size_t(c->cells) * 4, cudaMemcpyHostToDevice, c->st));
    return SL_OK;
}

sl_status sl_get_planes(sl_ctx* c, double* mean, void* hi, float* scale)
{
    sl_status s = planes_args(c, mean, hi, scale);
    if (s != SL_OK) return s;
    const Planes& p = c->planes[c->cur];
    const void* hb = hi_block(c, c->cur);
    if (c->nlo > 0)
        SL_CUDA(c, cudaMemcpy2DAsync(mean, size_t(c->cells) * 8, p.mean, size_t(c->pstride) * 8,
                                     size_t(c->cells) * 8, size_t(c->nlo), cudaMemcpyDeviceToHost, c->st));
    if (c->rec)
        SL_CUDA(c, cudaMemcpyAsync(hi, hb, size_t(c->cells) * c->rec * c->elem, cudaMemcpyDeviceToHost,
                                   c->st));
    else if (c->nhi > 0)
        SL_CUDA(c, cudaMemcpy2DAsync(hi, size_t(c->cells) * c->elem, hb, size_t(c->pstride) * c->elem,
                                     size_t(c->cells) * c->elem, size_t(c->nhi),
                                     cudaMemcpyDeviceToHost, c->st));
    if (p.scale)
        SL_CUDA(c, cudaMemcpyAsync(scale, p.scale, size_t(c->cells) * 4, cudaMemcpyDeviceToHost, c->st));
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    return SL_OK;
}

sl_status sl_project(sl_ctx* c, int nq, int nterms, const double* weights, const double* params)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (nq < 1 || nq > kMaxQuad) return fail(c, SL_EINVAL, "nq must be in 1..%d", kMaxQuad);
    if (nterms < 0 || (nterms > 0 && (!weights || !params))) return fail(c, SL_EINVAL, "bad terms");
    for (int i = 0; i < nterms; ++i)
        if (!std::isfinite(weights[i])) return fail(c, SL_ENAN, "non-finite weight");
    for (int i = 0; i < nterms * c->ndim * 4; ++i)
        if (!std::isfinite(params[i])) return fail(c, SL_ENAN, "non-finite factor parameter");
    ProjectArgs pa{};
    pa.ndim = c->ndim;
    pa.K = c->K;
    pa.nq = nq;
    pa.nterms = nterms;
    uint32_t nmax = 1;
    for (int m = 0; m < c->ndim; ++m) {
        pa.n[m] = uint32_t(c->g.n[m]);
        pa.lo[m] = c->g.lo[m];
        pa.h[m] = cell_width(c->g, m);
        nmax = std::max<uint32_t>(nmax, pa.n[m]);
    }
    // Gauss-Legendre nodes and weights: roots of P_nq by Newton's method.
    for (int i = 0; i < nq; ++i) {
        double z = std::cos(M_PI * (nq - i - 0.25) / (nq + 0.5));
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = z;
            for (int m = 2; m <= nq; ++m) {
                const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
                p0 = p1;
                p1 = p2;
            }
            const double dp = nq * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) <= 1e-17) break;
        }
        double p0 = 1.0, p1 = z;
        for (int m = 2; m <= nq; ++m) {
            const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
            p0 = p1;
            p1 = p2;
        }
        const double dp = nq * (z * p1 - p0) / (z * z - 1.0);
        pa.node[i] = z;
        pa.weight[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    const size_t tab_n = size_t(std::max(nterms, 1)) * c->ndim * nmax * c->O;
    const size_t need = (tab_n + size_t(std::max(nterms, 1)) * (1 + c->ndim * 4)) * 8;
    if (need > c->proj_bytes) {
        if (c->d_proj) {
            cudaStreamSynchronize(c->st);
            cudaFree(c->d_proj);
            c->d_proj = nullptr;
            c->proj_bytes = 0;
        }
        cudaError_t e = dev_malloc(reinterpret_cast<void**>(&c->d_proj), need);
        if (e != cudaSuccess) return fail(c, SL_ENOMEM, "projection workspace: %s", cudaGetErrorString(e));
        c->proj_bytes = need;
    }
    double* d_tab = c->d_proj;
    double* d_w = d_tab + tab_n;
    double* d_p = d_w + std::max(nterms, 1);
    if (nterms > 0) {
        SL_CUDA(c, cudaMemcpyAsync(d_w, weights, size_t(nterms) * 8, cudaMemcpyHostToDevice, c->st));
        SL_CUDA(c, cudaMemcpyAsync(d_p, params, size_t(nterms) * c->ndim * 4 * 8,
                                   cudaMemcpyHostToDevice, c->st));
    }
    SL_CUDA(c, launch_project(pa, d_w, d_p, d_tab, nmax, codec_of(c), uint32_t(c->cells), c->st));
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    return SL_OK;
}

sl_status sl_advect(sl_ctx* c, int dim, int shift_dim, const double* shifts, int64_t nshift)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (dim < 0 || dim >= c->ndim) return fail(c, SL_EINVAL, "dim %d out of range", dim);
    if (shift_dim < -1 || shift_dim >= c->ndim || shift_dim == dim)
        return fail(c, SL_EINVAL, "shift_dim %d invalid for dim %d", shift_dim, dim);
    const int64_t expect = shift_dim < 0 ? 1 : c->g.n[shift_dim];
    if (nshift != expect) return fail(c, SL_EINVAL, "nshift = %lld, expected %lld", (long long)nshift, (long long)expect);
    if (!shifts) return fail(c, SL_EINVAL, "shifts is NULL");
    for (int64_t i = 0; i < nshift; ++i)
        if (!std::isfinite(shifts[i]) || std::fabs(shifts[i]) > 1e15)
            return fail(c, SL_ENAN, "shift %lld is not finite or too large", (long long)i);
    if (c->capturing) return fail(c, SL_EINVAL, "sl_advect cannot be captured (host shifts)");
    SL_CUDA(c, cudaMemcpyAsync(c->d_shifts, shifts, size_t(nshift) * 8, cudaMemcpyHostToDevice, c->st));
    ShiftSource src{};
    src.kind = 0;
    src.data = c->d_shifts;
    sl_status s = build_table(c, dim, int(nshift), src);
    if (s != SL_OK) return s;
    return run_sweep(c, dim, shift_dim);
}

sl_status sl_set_fields(sl_ctx* c, const double* fields, int64_t count)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (count != c->nfields) return fail(c, SL_EINVAL, "count = %lld, expected %lld", (long long)count, (long long)c->nfields);
    if (count == 0) {
        c->fields_set = true;
        return SL_OK;
    }
    if (!fields) return fail(c, SL_EINVAL, "fields is NULL");
    for (int64_t i = 0; i < count; ++i)
        if (!std::isfinite(fields[i])) return fail(c, SL_ENAN, "non-finite field sample %lld", (long long)i);
    SL_CUDA(c, cudaMemcpyAsync(c->d_fields, fields, size_t(count) * 8, cudaMemcpyHostToDevice, c->st));
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    c->fields_set = true;
    return SL_OK;
}

// The grid's one x dimension and its v dimension, or -1 if the grid is not
// 1+1-dimensional with that one pair.
static bool vp_dims(const sl_ctx* c, int* x, int* v)
{
    if (c->ndim != 2) return false;
    for (int m = 0; m < 2; ++m)
        if (c->g.pair[m] == 1 - m && c->g.pair[1 - m] < 0) {
            *x = m;
            *v = 1 - m;
            return true;
        }
    return false;
}

static sl_status vp_alloc(sl_ctx* c)
{
    if (c->mode == M_F32ALL)
        return fail(c, SL_ENOTSUP, "the self-consistent field reads the FP64 mean plane, which SL_FP32 lacks");
    if (c->d_vp) return SL_OK;
    if (c->capturing) return fail(c, SL_EINVAL, "cannot allocate during a capture");
    const size_t nx = size_t(c->g.n[c->vp_x]);
    const size_t n = size_t(vp_chunks(uint32_t(c->g.n[c->vp_v]))) * nx + nx + 1;
    cudaError_t e = dev_malloc(reinterpret_cast<void**>(&c->d_vp), n * sizeof(double));
    if (e != cudaSuccess) {
        c->d_vp = nullptr;
        return fail(c, SL_ENOMEM, "cudaMalloc(%zu bytes): %s", n * sizeof(double), cudaGetErrorString(e));
    }
    return SL_OK;
}

sl_status sl_set_poisson(sl_ctx* c, int enable)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (!enable) {
        c->poisson = false;
        return SL_OK;
    }
    int x = -1, v = -1;
    if (!vp_dims(c, &x, &v)) return fail(c, SL_EINVAL, "the self-consistent field needs one x and one v dimension");
    c->vp_x = x;
    c->vp_v = v;
    sl_status s = vp_alloc(c);
    if (s != SL_OK) return s;
    c->poisson = true;
    return SL_OK;
}

// Node velocities of every x-dimension and the node tables, allocated once.
static sl_status nodal_alloc(sl_ctx* c)
{
    if (c->d_nodal) return SL_OK;
    if (c->capturing) return fail(c, SL_EINVAL, "cannot allocate during a capture");
    if (c->mode != M_FP64 && c->mode != M_F32)
        return fail(c, SL_ENOTSUP, "the nodal-in-velocity x-sweep takes the FP64 and mixed FP32 stores");
    NodalArgs tmp{};
    double eta[kMaxO], w[kMaxO];
    nodal_setup(c->K, eta, w, &tmp);
    std::vector<double> vel;
    int maxcls = 1, maxnv = 1;
    for (int m = 0; m < c->ndim; ++m) {
        const int p = c->g.pair[m];
        if (p < 0) continue;
        maxnv = std::max(maxnv, int(c->g.n[p]));
        c->nodal_vel_off[m] = int64_t(vel.size());
        const double hv = cell_width(c->g, p);
        for (int64_t j = 0; j < c->g.n[p]; ++j)
            for (int q = 0; q < c->O; ++q) vel.push_back(c->g.lo[p] + (double(j) + 0.5 + 0.5 * eta[q]) * hv);
        maxcls = std::max(maxcls, int(c->g.n[p] * c->O));
    }
    if (vel.empty()) return fail(c, SL_EINVAL, "the nodal-in-velocity x-sweep needs an x-dimension with a pair");
    const size_t A = 256;
    size_t off = align_up(vel.size() * 8, A);
    const size_t o_sig = off;
    off = align_up(off + size_t(maxcls) * 4, A);
    const size_t o_alpha = off;
    off = align_up(off + size_t(maxcls) * 8, A);
    const size_t o_ab64 = off;
    off = align_up(off + size_t(maxcls) * ab_stride64(c->O) * 8, A);
    const size_t o_ab32 = off;
    off = align_up(off + size_t(maxcls) * ab_stride32(c->O) * 4, A);
    const size_t o_abar = off;
    off = align_up(off + size_t(maxnv) * 8, A);
    const size_t o_na32 = off;
    off = align_up(off + size_t(maxnv) * kNa32 * 4, A);
    void* mem = nullptr;
    cudaError_t e = dev_malloc(&mem, off);
    if (e != cudaSuccess) return fail(c, SL_ENOMEM, "cudaMalloc(%zu bytes): %s", off, cudaGetErrorString(e));
    e = cudaMemcpy(mem, vel.data(), vel.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return cuda_fail(c, e, "node velocities");
    }
    char* b = static_cast<char*>(mem);
    c->d_nodal = mem;
    c->nodal_maxcls = maxcls;
    c->d_nsig = reinterpret_cast<int32_t*>(b + o_sig);
    c->d_nalpha = reinterpret_cast<double*>(b + o_alpha);
    c->d_nab64 = reinterpret_cast<double*>(b + o_ab64);
    c->d_nab32 = reinterpret_cast<float*>(b + o_ab32);
    c->d_nabar = reinterpret_cast<double*>(b + o_abar);
    c->d_nna32 = reinterpret_cast<float*>(b + o_na32);
    return SL_OK;
}

sl_status sl_set_nodal_velocity(sl_ctx* c, int enable)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (!enable) {
        c->nodal = false;
        return SL_OK;
    }
    if (c->ndim < 2) return fail(c, SL_EINVAL, "the nodal-in-velocity x-sweep needs an x-dimension with a pair");
    if (c->wide) return fail(c, SL_ENOTSUP, "the nodal-in-velocity x-sweep does not take SL_ARITH_FP64");
    sl_status s = nodal_alloc(c);
    if (s != SL_OK) return s;
    c->nodal = true;
    return SL_OK;
}

sl_status sl_advect_nodal(sl_ctx* c, int dim, double tau)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (dim < 0 || dim >= c->ndim || c->g.pair[dim] < 0)
        return fail(c, SL_EINVAL, "dim must be an x-dimension (pair[dim] >= 0)");
    if (!std::isfinite(tau)) return fail(c, SL_ENAN, "tau is not finite");
    if (c->wide) return fail(c, SL_ENOTSUP, "the nodal-in-velocity x-sweep does not take SL_ARITH_FP64");
    sl_status s = nodal_alloc(c);
    if (s != SL_OK) return s;
    s = nodal_table(c, dim, tau);
    if (s != SL_OK) return s;
    return run_sweep(c, dim, -1, true);
}

sl_status sl_set_arithmetic(sl_ctx* c, int arith)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (arith != SL_ARITH_STORE && arith != SL_ARITH_FP64) return fail(c, SL_EINVAL, "unknown arithmetic %d", arith);
    if (c->capturing) return fail(c, SL_EINVAL, "cannot change the arithmetic during a capture");
    if (c->mode == M_FP64) return SL_OK;   // already FP64 throughout
    if (arith == SL_ARITH_STORE) {
        c->wide = false;
        return SL_OK;
    }
    if (is_scaled(c)) return fail(c, SL_ENOTSUP, "SL_ARITH_FP64 takes the stores with FP32 planes");
    if (c->nodal) return fail(c, SL_ENOTSUP, "SL_ARITH_FP64 does not take nodal-in-velocity x-sweeps");
    c->wide = true;
    return SL_OK;
}

sl_status sl_field_energy(sl_ctx* c, double* energy)
{
    if (!c || !energy) return fail(nullptr, SL_EINVAL, "NULL argument");
    if (c->capturing) return fail(c, SL_EINVAL, "cannot read the field energy during a capture");
    int x = -1, v = -1;
    if (!vp_dims(c, &x, &v)) return fail(c, SL_EINVAL, "the self-consistent field needs one x and one v dimension");
    c->vp_x = x;
    c->vp_v = v;
    sl_status s = vp_alloc(c);
    if (s != SL_OK) return s;
    const size_t nx = size_t(c->g.n[x]);
    double* E = c->d_vp + size_t(vp_chunks(uint32_t(c->g.n[v]))) * nx;
    SL_CUDA(c, vp_field(c, E, E + nx));
    SL_CUDA(c, cudaMemcpyAsync(c->h_mass, E + nx, 8, cudaMemcpyDeviceToHost, c->st));
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    *energy = c->h_mass[0];
    return SL_OK;
}

sl_status sl_get_field(sl_ctx* c, double* field)
{
    if (!c || !field) return fail(nullptr, SL_EINVAL, "NULL argument");
    if (c->capturing) return fail(c, SL_EINVAL, "cannot read the field during a capture");
    int x = -1, v = -1;
    if (!vp_dims(c, &x, &v)) return fail(c, SL_EINVAL, "the self-consistent field needs one x and one v dimension");
    c->vp_x = x;
    c->vp_v = v;
    sl_status s = vp_alloc(c);
    if (s != SL_OK) return s;
    const size_t nx = size_t(c->g.n[x]);
    double* E = c->d_vp + size_t(vp_chunks(uint32_t(c->g.n[v]))) * nx;
    SL_CUDA(c, vp_field(c, E, nullptr));
    SL_CUDA(c, cudaMemcpyAsync(field, E, nx * 8, cudaMemcpyDeviceToHost, c->st));
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    return SL_OK;
}

static sl_status check_step_args(sl_ctx* c, sl_splitting sp, double dt, int nsteps)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (sp != SL_LIE && sp != SL_STRANG) return fail(c, SL_EINVAL, "unknown splitting %d", int(sp));
    if (!std::isfinite(dt)) return fail(c, SL_ENAN, "dt is not finite");
    if (nsteps < 0) return fail(c, SL_EINVAL, "nsteps < 0");
    bool any = false;
    for (int m = 0; m < c->ndim; ++m) any |= c->g.pair[m] >= 0;
    if (!any) return fail(c, SL_EINVAL, "grid has no x/v pairs to split");
    if (c->nfields > 0 && !c->fields_set && !c->poisson)
        return fail(c, SL_EINVAL, "fields not set (sl_set_fields or sl_set_poisson)");
    return SL_OK;
}

sl_status sl_step(sl_ctx* c, sl_splitting sp, double dt, int nsteps)
{
    sl_status s = check_step_args(c, sp, dt, nsteps);
    if (s != SL_OK) return s;
    NvtxRange range("sl_step");
    return enqueue_steps(c, sp, dt, nsteps);
}

sl_status sl_mass(sl_ctx* c, double* out)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (!out) return fail(c, SL_EINVAL, "out is NULL");
    double vol = 1.0;
    for (int m = 0; m < c->ndim; ++m) vol *= cell_width(c->g, m);
    if (c->mode == M_F32ALL)   // the mean is FP32 plane 0
        SL_CUDA(c, launch_mass_f32(static_cast<const float*>(hi_block(c, c->cur)), uint32_t(c->cells),
                                   c->d_partials, c->mass_nblk, vol, c->d_mass, c->st));
    else
        SL_CUDA(c, launch_mass(c->planes[c->cur].mean, uint32_t(c->cells), c->d_partials, c->mass_nblk,
                               vol, c->d_mass, c->st));
    SL_CUDA(c, cudaMemcpyAsync(c->h_mass, c->d_mass, 8, cudaMemcpyDeviceToHost, c->st));
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    *out = *c->h_mass;
    return SL_OK;
}

sl_status sl_graph_capture(sl_ctx* c, sl_splitting sp, double dt, int nsteps)
{
    sl_status s = check_step_args(c, sp, dt, nsteps);
    if (s != SL_OK) return s;
    const int sweeps = int(plan_of(c, sp).size()) * nsteps;
    return capture_graphs(c, sweeps, [&]() { return enqueue_steps(c, sp, dt, nsteps); });
}

sl_status sl_graph_capture_advect(sl_ctx* c, int dim, int shift_dim, const double* shifts, int64_t nshift,
                                  int nsteps)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (dim < 0 || dim >= c->ndim) return fail(c, SL_EINVAL, "dim %d out of range", dim);
    if (shift_dim < -1 || shift_dim >= c->ndim || shift_dim == dim)
        return fail(c, SL_EINVAL, "shift_dim %d invalid for dim %d", shift_dim, dim);
    const int64_t expect = shift_dim < 0 ? 1 : c->g.n[shift_dim];
    if (nshift != expect) return fail(c, SL_EINVAL, "nshift = %lld, expected %lld", (long long)nshift, (long long)expect);
    if (!shifts) return fail(c, SL_EINVAL, "shifts is NULL");
    if (nsteps < 1) return fail(c, SL_EINVAL, "nsteps < 1");
    for (int64_t i = 0; i < nshift; ++i)
        if (!std::isfinite(shifts[i]) || std::fabs(shifts[i]) > 1e15)
            return fail(c, SL_ENAN, "shift %lld is not finite or too large", (long long)i);
    if (c->capturing) return fail(c, SL_EINVAL, "already capturing");
    // the graph's own copy of the shifts, so later calls cannot change what it reads
    if (c->gshifts_n < nshift) {
        if (c->d_gshifts) cudaFree(c->d_gshifts);
        c->d_gshifts = nullptr;
        c->gshifts_n = 0;
        cudaError_t e = dev_malloc(reinterpret_cast<void**>(&c->d_gshifts), size_t(nshift) * 8);
        if (e != cudaSuccess) return fail(c, SL_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
        c->gshifts_n = nshift;
    }
    SL_CUDA(c, cudaMemcpyAsync(c->d_gshifts, shifts, size_t(nshift) * 8, cudaMemcpyHostToDevice, c->st));
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    // a short 1D line of the FP64 store with one shift: every step in one
    // cluster launch (sl_sweep_1d.cu), each step building its matrices
    const bool one_launch = c->ndim == 1 && c->mode == M_FP64 && !c->wide && shift_dim < 0 &&
                            sweep_1d_cluster_ok(c->K, uint32_t(c->g.n[0]));
    return capture_graphs(c, nsteps, [&]() -> sl_status {
        if (one_launch) {
            cudaError_t e = launch_sweep_1d_cluster(c->K, c->planes[c->cur], c->planes[c->cur ^ (nsteps & 1)],
                                                    c->pstride, uint32_t(c->g.n[0]), c->d_gshifts, c->poly,
                                                    nsteps, c->st);
            if (e != cudaSuccess) return cuda_fail(c, e, "1D cluster sweep launch");
            c->cur ^= nsteps & 1;
            return SL_OK;
        }
        for (int q = 0; q < nsteps; ++q) {
            ShiftSource src{};
            src.kind = 0;
            src.data = c->d_gshifts;
            sl_status r = build_table(c, dim, int(nshift), src);
            if (r != SL_OK) return r;
            r = run_sweep(c, dim, shift_dim);
            if (r != SL_OK) return r;
        }
        return SL_OK;
    });
}

sl_status sl_graph_launch(sl_ctx* c)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (c->graph_start < 0) return fail(c, SL_EINVAL, "no graph captured");
    const int gi = c->cur == c->graph_start ? 0 : 1;
    if (!c->gexec[gi]) return fail(c, SL_EINVAL, "no graph for the current buffer parity");
    SL_CUDA(c, cudaGraphLaunch(c->gexec[gi], c->st));
    c->cur ^= c->graph_flip;
    return SL_OK;
}

sl_status sl_synchronize(sl_ctx* c)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    return SL_OK;
}

sl_status sl_profile_dims(const sl_ctx* c, int64_t* launches, double* ms)
{
    if (!c || !launches || !ms) return fail(nullptr, SL_EINVAL, "NULL argument");
    for (int m = 0; m < SL_MAX_DIM; ++m) {
        launches[m] = c->last_dim_launches[m];
        ms[m] = c->last_dim_ms[m];
    }
    return SL_OK;
}

sl_status sl_get_tune(const sl_ctx* c, int dim, sl_tune* out)
{
    if (!c || !out) return fail(nullptr, SL_EINVAL, "NULL argument");
    if (dim < 0 || dim >= c->ndim) return fail(const_cast<sl_ctx*>(c), SL_EINVAL, "dim out of range");
    const auto& t = c->tune[dim];
    out->block = t.block;
    out->fibres_per_thread = t.ft;
    out->unroll = t.unroll;
    out->pipeline = t.pipeline;
    out->max_blocks_per_sm = t.occ;
    out->reserved = 0;
    out->chunk = dim == 0 && !c->rec ? 0 : int64_t(t.chunk);
    return SL_OK;
}

static sl_status check_tune(sl_ctx* c, int dim, const sl_tune* t)
{
    const bool lanes = rec_lanes(c, t->fibres_per_thread);
    const int maxb = (dim == 0 && !c->rec) || lanes ? 256 : 128;
    if (t->reserved != 0) return fail(c, SL_EINVAL, "sl_tune.reserved must be 0");
    if (is_split(c)) {
        if (t->fibres_per_thread != 1) return fail(c, SL_EINVAL, "the # double = 2, 3 stores take one fibre per thread");
        if (t->pipeline != 0 || t->max_blocks_per_sm != 0)
            return fail(c, SL_EINVAL, "the # double = 2, 3 stores have no pipeline or block limit");
        if (dim == 0 && t->unroll != 1) return fail(c, SL_EINVAL, "unroll along dimension 0 must be 1");
        if (dim > 0 && t->unroll != 1 && t->unroll != 2) return fail(c, SL_EINVAL, "unroll must be 1 or 2");
    }
    if (t->max_blocks_per_sm != 0) {
        if (t->max_blocks_per_sm < 4 || t->max_blocks_per_sm > 6)
            return fail(c, SL_EINVAL, "max_blocks_per_sm must be 0, 4, 5 or 6");
        if (is_scaled(c) || dim == 0 || t->pipeline != 0)
            return fail(c, SL_EINVAL, "max_blocks_per_sm applies to the register walk of the FP64/FP32 stores");
    }
    if (t->block < 32 || t->block > maxb || t->block % 32)
        return fail(c, SL_EINVAL, "block must be a multiple of 32 in [32, %d]", maxb);
    if (!is_scaled(c)) {
        if (t->fibres_per_thread > c->nfib)
            return fail(c, SL_EINVAL, "fibres_per_thread %d exceeds the %lld fibres of a cell",
                        t->fibres_per_thread, (long long)c->nfib);
        if (dim == 0 && t->unroll == 1 && !unit_ft_ok(t->fibres_per_thread))
            return fail(c, SL_EINVAL, "fibres_per_thread %d not provided along dimension 0",
                        t->fibres_per_thread);
        if (dim == 0 && t->unroll != 1) {
            if (t->unroll != unit_vec_width(c))
                return fail(c, SL_EINVAL, "unroll along dimension 0 must be 1 or %d (n_0 divisible by it)",
                            int(16 / c->elem));
            if (t->fibres_per_thread < 1 || t->fibres_per_thread > 4)
                return fail(c, SL_EINVAL, "the vector form takes 1..4 fibres per thread");
        }
        if (dim > 0 && t->pipeline == 0 && !strided_ok(t->fibres_per_thread, t->unroll))
            return fail(c, SL_EINVAL, "(fibres_per_thread %d, unroll %d) not provided",
                        t->fibres_per_thread, t->unroll);
        if (dim > 0 && t->pipeline != 0 && !async_ok(t->fibres_per_thread, t->pipeline))
            return fail(c, SL_EINVAL, "(fibres_per_thread %d, pipeline %d) not provided",
                        t->fibres_per_thread, t->pipeline);
        if (dim > 0 && t->pipeline != 0 && t->block != 64 && t->block != 128)
            return fail(c, SL_EINVAL, "the cp.async walk runs with 64 or 128 threads per block");
        if (dim == 0 && t->pipeline != 0) return fail(c, SL_EINVAL, "pipeline applies to dimensions > 0");
    } else {
        if (t->pipeline != 0) return fail(c, SL_EINVAL, "the scaled stores have no cp.async pipeline");
        const std::vector<int> ok = scaled_fts(c);
        if (std::find(ok.begin(), ok.end(), t->fibres_per_thread) == ok.end())
            return fail(c, SL_EINVAL, "fibres_per_thread %d is not a provided split of the %lld fibres",
                        t->fibres_per_thread, (long long)c->nfib);
    }
    if (c->rec && lanes) {
        if (t->unroll != 1 && t->unroll != 2 && t->unroll != 4)
            return fail(c, SL_EINVAL, "lane-group record sweeps take unroll 1, 2 or 4");
        if (dim == 0 && (t->chunk < 1 || t->chunk > c->g.n[0]))
            return fail(c, SL_EINVAL, "lane-group record sweeps walk dimension 0 too: chunk in [1, n_0]");
    } else if (c->rec) {
        if (t->unroll != 1 && t->unroll != 2)
            return fail(c, SL_EINVAL, "record sweeps take unroll 1 (plain) or 2 (prefetching walk)");
        if (dim == 0 && t->chunk != 0 && (t->chunk < 1 || t->chunk > c->g.n[0]))
            return fail(c, SL_EINVAL, "chunk along dimension 0 must be 0 (one thread per cell) or in [1, n_0]");
    }
    if (c->rec && dim == 0 && t->chunk > 0 && (c->g.n[0] + t->chunk - 1) / t->chunk > 65535)
        return fail(c, SL_EINVAL, "too many chunks for one launch");
    if (dim > 0) {
        const int64_t N = c->g.n[dim];
        if (t->chunk < 1 || t->chunk > N) return fail(c, SL_EINVAL, "chunk must be in [1, n_dim]");
        const int ft = is_scaled(c) ? 1 : t->fibres_per_thread;
        if (((N + t->chunk - 1) / t->chunk) * fibre_groups(c, ft) > 65535)
            return fail(c, SL_EINVAL, "too many chunks x fibre groups for one launch");
    }
    return SL_OK;
}

sl_status sl_set_tune(sl_ctx* c, int dim, const sl_tune* t)
{
    if (!c || !t) return fail(nullptr, SL_EINVAL, "NULL argument");
    if (dim < 0 || dim >= c->ndim) return fail(c, SL_EINVAL, "dim out of range");
    sl_status s = check_tune(c, dim, t);
    if (s != SL_OK) return s;
    auto& d = c->tune[dim];
    d.block = t->block;
    d.ft = t->fibres_per_thread;
    d.unroll = is_scaled(c) && !c->rec ? 1 : t->unroll;
    d.pipeline = is_scaled(c) || dim == 0 ? 0 : t->pipeline;
    d.occ = t->max_blocks_per_sm;
    d.chunk = dim == 0 && !c->rec ? 0 : uint32_t(t->chunk);
    return SL_OK;
}

sl_status sl_autotune(sl_ctx* c, int reps)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    if (c->capturing) return fail(c, SL_EINVAL, "cannot autotune during a capture");
    if (reps < 1) reps = 1;
    if (reps > 50) reps = 50;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SL_CUDA(c, cudaEventCreate(&e0));
    SL_CUDA(c, cudaEventCreate(&e1));
    sl_status result = SL_OK;
    for (int m = 0; m < c->ndim && result == SL_OK; ++m) {
        const int sd = natural_shift_dim(c, m);
        const int nclass = sd < 0 ? 1 : int(c->g.n[sd]);
        // shifts of -0.63, 0.37 and 1.37 cells in turn over the classes, so
        // that, as in a real step, sigma differs between neighbouring lines
        // whose class follows their own coordinate
        std::vector<double> sh(static_cast<size_t>(nclass));
        for (int q = 0; q < nclass; ++q) sh[size_t(q)] = 0.37 + double(q % 3) - 1.0;
        cudaError_t e = cudaMemcpyAsync(c->d_shifts, sh.data(), sh.size() * 8, cudaMemcpyHostToDevice, c->st);
        if (e != cudaSuccess) {
            result = cuda_fail(c, e, "autotune shifts");
            break;
        }
        ShiftSource src{};
        src.kind = 0;
        src.data = c->d_shifts;
        result = build_table(c, m, nclass, src);
        if (result != SL_OK) break;

        std::vector<sl_ctx::Tune> cand;
        if (is_scaled(c)) {
            const uint32_t ch = chunk_for(c, m, 1, 1);
            for (int f : scaled_fts(c)) {
                if (rec_lanes(c, f)) {   // lane groups walk every dimension
                    const uint32_t chl = chunk_for(c, m, 1, c->rec / 16);
                    for (int u : {1, 2, 4})
                        for (int b : {128, 256}) cand.push_back({b, f, u, chl, 0});
                } else if (f == c->nfib && c->rec) {
                    if (m == 0)
                        for (int b : {64, 128}) cand.push_back({b, f, 1, 0, 0});
                    for (int u : {1, 2})
                        for (int b : {64, 128}) cand.push_back({b, f, u, ch, 0});
                } else if (f == c->nfib) {
                    for (int b : {64, 128, 256})
                        if (m == 0 || b <= 128) cand.push_back({b, f, 1, m == 0 ? 0u : ch, 0});
                } else {   // a cooperative split of the cell's fibres
                    cand.push_back({128, f, 1, m == 0 ? 0u : ch, 0});
                }
            }
        } else if (is_split(c)) {
            if (m == 0)
                for (int b : {128, 256}) cand.push_back({b, 1, 1, 0, 0});
            else
                for (int u : {1, 2})
                    for (int b : {64, 128}) cand.push_back({b, 1, u, chunk_for(c, m, 1, 1), 0});
        } else if (m == 0) {
            {
                for (int ft : {1, 2, 3, 4, 9})
                    if (ft <= c->nfib)
                        for (int b : {128, 256}) cand.push_back({b, ft, 1, 0, 0});
                if (const int v = unit_vec_width(c))
                    for (int ft : {1, 2, 3, 4})
                        if (ft <= c->nfib)
                            for (int b : {128, 256}) cand.push_back({b, ft, v, 0, 0});
            }
        } else {
            {
                const int fu[][2] = {{1, 1}, {1, 2}, {1, 4}, {2, 1}, {2, 2}, {2, 4}, {3, 1}, {3, 2}};
                for (auto& x : fu)
                    if (x[0] <= c->nfib)
                        for (int occ : {0, 5, 4}) {
                            sl_ctx::Tune t{128, x[0], x[1], chunk_for(c, m, x[0], 1), 0};
                            t.occ = occ;
                            cand.push_back(t);
                        }
                const int fp[][2] = {{1, 4}, {1, 8}, {2, 4}, {2, 8}, {3, 4}};
                for (auto& x : fp)
                    if (x[0] <= c->nfib)
                        for (int b : {64, 128})
                            cand.push_back({b, x[0], 1, chunk_for(c, m, x[0], 1), x[1]});
            }
        }
        const sl_ctx::Tune keep = c->tune[m];
        // time one candidate: a warm-up launch, then reps launches
        auto time_one = [&](const sl_ctx::Tune& t, float* ms) {
            c->tune[m] = t;
            cudaError_t err = launch_only(c, m, sd);
            if (err == cudaSuccess) err = cudaEventRecord(e0, c->st);
            for (int r = 0; r < reps && err == cudaSuccess; ++r) err = launch_only(c, m, sd);
            if (err == cudaSuccess) err = cudaEventRecord(e1, c->st);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
            return err;
        };
        std::vector<float> t_ms(cand.size(), 1e30f);
        for (size_t q = 0; q < cand.size() && e == cudaSuccess; ++q) e = time_one(cand[q], &t_ms[q]);
        // second round over the three fastest, keeping each one's better time
        std::vector<size_t> order(cand.size());
        for (size_t q = 0; q < order.size(); ++q) order[q] = q;
        std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return t_ms[x] < t_ms[y]; });
        for (size_t r = 0; r < std::min<size_t>(3, order.size()) && e == cudaSuccess; ++r) {
            float ms = 1e30f;
            e = time_one(cand[order[r]], &ms);
            t_ms[order[r]] = std::min(t_ms[order[r]], ms);
        }
        if (e != cudaSuccess) {
            c->tune[m] = keep;
            result = cuda_fail(c, e, "autotune launch");
            break;
        }
        size_t best = 0;
        for (size_t q = 1; q < cand.size(); ++q)
            if (t_ms[q] < t_ms[best]) best = q;
        c->tune[m] = cand.empty() ? keep : cand[best];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return result;
}

sl_status sl_profile_enable(sl_ctx* c, int enable)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    c->prof = enable != 0;
    return SL_OK;
}

sl_status sl_profile_query(sl_ctx* c, int64_t* launches, double* ms, double* bytes)
{
    if (!c) return fail(nullptr, SL_EINVAL, "ctx is NULL");
    SL_CUDA(c, cudaStreamSynchronize(c->st));
    double tot = 0.0;
    for (int m = 0; m < SL_MAX_DIM; ++m) {
        c->last_dim_launches[m] = 0;
        c->last_dim_ms[m] = 0.0;
    }
    for (size_t q = 0; q < c->ev_used.size(); ++q) {
        auto& pr = c->ev_used[q];
        float t = 0.0f;
        SL_CUDA(c, cudaEventElapsedTime(&t, pr.first, pr.second));
        tot += t;
        c->last_dim_launches[c->ev_dim[q]]++;
        c->last_dim_ms[c->ev_dim[q]] += t;
        c->ev_free.push_back(pr.first);
        c->ev_free.push_back(pr.second);
    }
    c->ev_used.clear();
    c->ev_dim.clear();
    if (launches) *launches = c->prof_launches;
    if (ms) *ms = tot;
    if (bytes) *bytes = 2.0 * double(c->state_bytes) * double(c->prof_launches);
    c->prof_launches = 0;
    return SL_OK;
}

}  // extern "C"
