// sl_batch_api.cu -- host side of the batched API (sl_batch_* in sl.h).
//
// A batch owns one single-problem context per problem (each with its own
// ping-pong state, tables and fields).  All problems advance together: every
// split substep is one table launch over all problems and one persistent
// sweep launch over a work list of tiles of all problems, so uneven problem
// sizes balance across the GPU (along dimensions > 0 the tiles are sorted by
// decreasing cost and taken from a shared counter).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sl_host.h"

using namespace sl;
using namespace sl::host;

struct sl_batch {
    std::vector<sl_ctx*> probs;
    int nprob = 0;
    int ndim = 0;
    sl::Mode mode = sl::M_F32;
    cudaStream_t st = nullptr;
    std::string err;
    int parity = 0;   // copy every problem currently reads
    int64_t state_bytes = 0;
    int sms = 1;

    // device arrays (one allocation)
    void* mem = nullptr;
    SweepArgs* d_args = nullptr;   // [dim][parity][prob]
    int32_t* d_kdeg = nullptr;     // [prob]
    BatchAB* d_ab = nullptr;       // [dim][prob]
    PolyTab* d_tabs = nullptr;     // [degree 0..3]
    BatchMass* d_mass_desc = nullptr;
    double* d_mass = nullptr;      // [prob]
    uint32_t* d_ctr = nullptr;     // [dim] work-list counters
    std::vector<double> h_mass;
    int maxcls[SL_MAX_DIM] = {0};

    // work lists per dimension
    BatchItem* d_items[SL_MAX_DIM] = {nullptr};
    int nitems[SL_MAX_DIM] = {0};
    struct Tune {
        int ft = 1;       // most fibres per thread (each problem takes min(ft, its fibres))
        int unroll = 1;   // cells per walk step (dimensions > 0), cells per thread (dimension 0)
        int rows = 64;    // rows per work item (dimensions > 0)
        int reps = 4;     // cell tiles per work item (dimension 0)
    } tune[SL_MAX_DIM];

    // side stream of the v-dimensions' table builds (see batch_steps)
    cudaStream_t st_tab = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int graph_start = -1;
    int graph_flip = 0;
    bool capturing = false;

    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    std::vector<int> ev_dim;
    int64_t prof_launches = 0;
    int64_t last_dim_launches[SL_MAX_DIM] = {0};
    double last_dim_ms[SL_MAX_DIM] = {0.0};
};

namespace {

sl_status bfail(sl_batch* b, sl_status s, const char* msg)
{
    if (b)
        b->err = msg;
    else
        fail(nullptr, s, "%s", msg);
    return s;
}

sl_status bcuda(sl_batch* b, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return bfail(b, SL_ECUDA, m.c_str());
}

#define SLB_CUDA(b, call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return bcuda((b), e_, #call); \
    } while (0)


// Work items and sweep geometry of dimension m for the batch's current tune.
sl_status rebuild_dim(sl_batch* b, int m)
{
    const auto& t = b->tune[m];
    std::vector<BatchItem> items;
    std::vector<int64_t> cost;   // values one item's threads update (dimensions > 0)
    std::vector<SweepArgs> args(2 * size_t(b->nprob));
    for (int p = 0; p < b->nprob; ++p) {
        sl_ctx* c = b->probs[p];
        c->tune[m].ft = int(std::min<int64_t>(t.ft, c->nfib));
        c->tune[m].unroll = t.unroll;
        c->tune[m].pipeline = 0;
        const int64_t N = c->g.n[m];
        c->tune[m].chunk = m == 0 ? 0 : uint32_t(std::min<int64_t>(N, t.rows));
        const int sd = natural_shift_dim(c, m);
        for (int par = 0; par < 2; ++par) args[size_t(par) * b->nprob + p] = make_args_parity(c, m, sd, par);
        const SweepArgs& a = args[p];
        const uint32_t nfg = uint32_t(a.nfg);
        if (m == 0) {
            const uint32_t span = uint32_t(kBatchBlock * t.reps * t.unroll);   // unroll: cells per thread
            const uint32_t tiles = (a.cells + span - 1) / span;
            for (uint32_t i = 0; i < tiles; ++i)   // the groups of a tile side by side (see unit_grid)
                for (uint32_t g = 0; g < nfg; ++g) items.push_back({uint32_t(p), i * span, g, 0});
        } else {
            const uint32_t tiles = (a.lines + kBatchLines - 1) / kBatchLines;
            const uint32_t nchunk = (a.N + a.chunk - 1) / a.chunk;
            const int64_t ft = c->tune[m].ft;
            for (uint32_t g = 0; g < nfg; ++g)
                for (uint32_t ch = 0; ch < nchunk; ++ch)
                    for (uint32_t i = 0; i < tiles; ++i) {
                        items.push_back({uint32_t(p), i * kBatchLines, g, ch});
                        const int64_t lines = std::min<int64_t>(kBatchLines, int64_t(a.lines) - int64_t(i) * kBatchLines);
                        const int64_t rows = std::min<int64_t>(a.chunk, int64_t(a.N) - int64_t(ch) * a.chunk);
                        const int64_t fib = std::min<int64_t>(ft, c->nfib - int64_t(g) * ft);
                        cost.push_back(lines * rows * fib * c->O);
                    }
        }
    }
    if (m > 0) {   // longest first (the blocks take them in order)
        std::vector<size_t> order(items.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
        std::vector<BatchItem> sorted(items.size());
        for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
        items.swap(sorted);
    }
    SLB_CUDA(b, cudaMemcpyAsync(b->d_args + size_t(m) * 2 * b->nprob, args.data(),
                                args.size() * sizeof(SweepArgs), cudaMemcpyHostToDevice, b->st));
    if (b->d_items[m]) {
        SLB_CUDA(b, cudaStreamSynchronize(b->st));
        cudaFree(b->d_items[m]);
        b->d_items[m] = nullptr;
    }
    if (dev_malloc(reinterpret_cast<void**>(&b->d_items[m]), std::max<size_t>(1, items.size()) * sizeof(BatchItem)) !=
        cudaSuccess)
        return bfail(b, SL_ENOMEM, "work list allocation");
    SLB_CUDA(b, cudaMemcpyAsync(b->d_items[m], items.data(), items.size() * sizeof(BatchItem),
                                cudaMemcpyHostToDevice, b->st));
    SLB_CUDA(b, cudaStreamSynchronize(b->st));
    b->nitems[m] = int(items.size());
    return SL_OK;
}

cudaEvent_t new_event()
{
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}

// Shift tables of every problem's dimension m over tau on stream st.
sl_status batch_tables(sl_batch* b, int m, double tau, cudaStream_t st)
{
    SLB_CUDA(b, launch_batch_ab(b->d_ab + size_t(m) * b->nprob, b->d_tabs, b->nprob, b->maxcls[m], tau, st));
    return SL_OK;
}

// The sweep of every problem along m with the tables already built.
sl_status batch_sweep(sl_batch* b, int m)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool prof = b->prof && !b->capturing;
    if (prof) {
        e0 = new_event();
        e1 = new_event();
        if (!e0 || !e1) return bfail(b, SL_ECUDA, "cudaEventCreate failed");
        SLB_CUDA(b, cudaEventRecord(e0, b->st));
    }
    const auto& t = b->tune[m];
    const int blocks = b->sms * batch_sweep_occupancy(b->mode, t.ft, t.unroll, m == 0);
    SLB_CUDA(b, launch_batch_sweep(b->mode, t.ft, t.unroll,
                                   b->d_args + (size_t(m) * 2 + b->parity) * b->nprob, b->d_kdeg,
                                   b->d_items[m], b->nitems[m], m == 0, t.reps, blocks, b->d_ctr + m,
                                   b->st));
    if (prof) {
        SLB_CUDA(b, cudaEventRecord(e1, b->st));
        b->ev.emplace_back(e0, e1);
        b->ev_dim.push_back(m);
        b->prof_launches++;
    }
    b->parity ^= 1;
    for (auto* c : b->probs) c->cur = b->parity;
    return SL_OK;
}

// The split steps.  As for one problem, a table depends on its dimension,
// tau and the fields only, so each dimension's tables are built once per
// step: the x-dimensions' before the step's first sweep, the v-dimensions'
// on the side stream while the x-sweeps run (joined before the first
// v-sweep); Strang's second x half-step reuses the first one's.
sl_status batch_steps(sl_batch* b, sl_splitting sp, double dt, int nsteps)
{
    const std::vector<SubStep> plan = plan_of(b->probs[0], sp);
    const sl_ctx* c0 = b->probs[0];
    bool ahead = true;
    for (const SubStep& x : plan)
        for (const SubStep& y : plan)
            if (x.dim == y.dim && x.frac != y.frac) ahead = false;
    for (int s = 0; s < nsteps; ++s) {
        bool built[SL_MAX_DIM] = {false};
        bool joined = true;
        if (ahead) {
            bool any_v = false;
            for (const SubStep& ss : plan) {
                if (c0->g.pair[ss.dim] < 0) {
                    any_v = true;
                } else if (!built[ss.dim]) {
                    sl_status r = batch_tables(b, ss.dim, ss.frac * dt, b->st);
                    if (r != SL_OK) return r;
                    built[ss.dim] = true;
                }
            }
            if (any_v) {
                SLB_CUDA(b, cudaEventRecord(b->ev_fork, b->st));
                SLB_CUDA(b, cudaStreamWaitEvent(b->st_tab, b->ev_fork, 0));
                for (const SubStep& ss : plan) {
                    if (c0->g.pair[ss.dim] >= 0 || built[ss.dim]) continue;
                    sl_status r = batch_tables(b, ss.dim, ss.frac * dt, b->st_tab);
                    if (r != SL_OK) return r;
                    built[ss.dim] = true;
                }
                SLB_CUDA(b, cudaEventRecord(b->ev_join, b->st_tab));
                joined = false;
            }
        }
        for (const SubStep& ss : plan) {
            if (!built[ss.dim]) {
                sl_status r = batch_tables(b, ss.dim, ss.frac * dt, b->st);
                if (r != SL_OK) return r;
            } else if (!joined && c0->g.pair[ss.dim] < 0) {
                SLB_CUDA(b, cudaStreamWaitEvent(b->st, b->ev_join, 0));
                joined = true;
            }
            sl_status r = batch_sweep(b, ss.dim);
            if (r != SL_OK) return r;
        }
        if (!joined) SLB_CUDA(b, cudaStreamWaitEvent(b->st, b->ev_join, 0));
    }
    return SL_OK;
}

sl_status check_prob(sl_batch* b, int p)
{
    if (!b) return fail(nullptr, SL_EINVAL, "batch is NULL");
    if (p < 0 || p >= b->nprob) return bfail(b, SL_EINVAL, "problem index out of range");
    return SL_OK;
}

sl_status forward(sl_batch* b, sl_ctx* c, sl_status s)
{
    if (s != SL_OK) b->err = c->err;
    return s;
}

void drop_graph(sl_batch* b)
{
    for (auto& g : b->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    b->graph_start = -1;
}

sl_status check_steps(sl_batch* b, sl_splitting sp, double dt, int nsteps)
{
    if (!b) return fail(nullptr, SL_EINVAL, "batch is NULL");
    if (sp != SL_LIE && sp != SL_STRANG) return bfail(b, SL_EINVAL, "unknown splitting");
    if (!std::isfinite(dt)) return bfail(b, SL_ENAN, "dt is not finite");
    if (nsteps < 0) return bfail(b, SL_EINVAL, "nsteps < 0");
    for (auto* c : b->probs)
        if (c->nfields > 0 && !c->fields_set) return bfail(b, SL_EINVAL, "fields not set (sl_batch_set_fields)");
    return SL_OK;
}

}  // namespace

extern "C" {

sl_status sl_batch_create(int nprob, const sl_grid* grids, const int* degrees, sl_storage storage,
                          void* cuda_stream, sl_batch** out)
{
    if (!out) return fail(nullptr, SL_EINVAL, "out is NULL");
    *out = nullptr;
    if (nprob < 1 || nprob > 65535) return fail(nullptr, SL_EINVAL, "nprob must be in 1..65535");
    if (!grids || !degrees) return fail(nullptr, SL_EINVAL, "grids or degrees is NULL");
    if (storage != SL_FP64 && storage != SL_MIX_FP32)
        return fail(nullptr, SL_ENOTSUP, "batches support the FP64 and mixed FP32 stores");
    bool any_pair = false;
    for (int p = 0; p < nprob; ++p) {
        sl_status s = check_grid(&grids[p], degrees[p], storage, nullptr);
        if (s != SL_OK) return s;
        if (degrees[p] > kBatchMaxK) return fail(nullptr, SL_ENOTSUP, "batched degrees are 0..%d", kBatchMaxK);
        if (grids[p].ndim != grids[0].ndim) return fail(nullptr, SL_EINVAL, "problems differ in ndim");
        for (int m = 0; m < grids[0].ndim; ++m)
            if (grids[p].pair[m] != grids[0].pair[m])
                return fail(nullptr, SL_EINVAL, "problems differ in their x/v pairing");
    }
    for (int m = 0; m < grids[0].ndim; ++m) any_pair |= grids[0].pair[m] >= 0;
    if (!any_pair) return fail(nullptr, SL_EINVAL, "batched problems need x/v pairs to split");

    sl_batch* b = new (std::nothrow) sl_batch();
    if (!b) return fail(nullptr, SL_ENOMEM, "host allocation failed");
    b->nprob = nprob;
    b->ndim = grids[0].ndim;
    b->mode = sl::Mode(storage);
    b->st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        delete b;
        return fail(nullptr, SL_ECUDA, "no CUDA device");
    }
    b->sms = prop.multiProcessorCount;
    auto cleanup = [&](sl_status s) {
        sl_batch_destroy(b);
        return s;
    };
    for (int p = 0; p < nprob; ++p) {
        sl_ctx* c = nullptr;
        sl_status s = sl_create(&grids[p], degrees[p], storage, cuda_stream, &c);
        if (s != SL_OK) return cleanup(s);
        b->probs.push_back(c);
        b->state_bytes += c->state_bytes;
        for (int m = 0; m < b->ndim; ++m) {
            const int sd = natural_shift_dim(c, m);
            b->maxcls[m] = std::max<int>(b->maxcls[m], sd < 0 ? 1 : int(c->g.n[sd]));
        }
    }
    // device arrays
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_args = take(sizeof(SweepArgs) * 2 * b->ndim * nprob);
    const size_t o_k = take(sizeof(int32_t) * nprob);
    const size_t o_ab = take(sizeof(BatchAB) * b->ndim * nprob);
    const size_t o_tabs = take(sizeof(PolyTab) * 4);
    const size_t o_md = take(sizeof(BatchMass) * nprob);
    const size_t o_m = take(sizeof(double) * nprob);
    const size_t o_ctr = take(sizeof(uint32_t) * SL_MAX_DIM);
    if (dev_malloc(&b->mem, off) != cudaSuccess) return cleanup(fail(nullptr, SL_ENOMEM, "batch tables"));
    char* base = static_cast<char*>(b->mem);
    b->d_args = reinterpret_cast<SweepArgs*>(base + o_args);
    b->d_kdeg = reinterpret_cast<int32_t*>(base + o_k);
    b->d_ab = reinterpret_cast<BatchAB*>(base + o_ab);
    b->d_tabs = reinterpret_cast<PolyTab*>(base + o_tabs);
    b->d_mass_desc = reinterpret_cast<BatchMass*>(base + o_md);
    b->d_mass = reinterpret_cast<double*>(base + o_m);
    b->d_ctr = reinterpret_cast<uint32_t*>(base + o_ctr);
    b->h_mass.resize(nprob);
    if (cudaStreamCreateWithFlags(&b->st_tab, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(fail(nullptr, SL_ECUDA, "batch side stream"));

    std::vector<int32_t> kd(nprob);
    std::vector<BatchAB> ab(size_t(b->ndim) * nprob);
    std::vector<BatchMass> md(nprob);
    std::vector<PolyTab> tabs(4);
    for (int K = 0; K < 4; ++K) build_poly_table(K, &tabs[K]);
    for (int p = 0; p < nprob; ++p) {
        sl_ctx* c = b->probs[p];
        kd[p] = c->K;
        double vol = 1.0;
        for (int m = 0; m < c->ndim; ++m) vol *= cell_width(c->g, m);
        md[p] = BatchMass{{c->planes[0].mean, c->planes[1].mean}, uint32_t(c->cells), vol};
        for (int m = 0; m < b->ndim; ++m) {
            BatchAB& d = ab[size_t(m) * nprob + p];
            d.K = c->K;
            d.N = uint32_t(c->g.n[m]);
            d.sigma = c->d_sigma[m];
            d.alpha = c->d_alpha[m];
            d.ab64 = c->d_ab64[m];
            d.ab32 = c->d_ab32[m];
            d.h = cell_width(c->g, m);
            if (c->g.pair[m] >= 0) {
                const int v = c->g.pair[m];
                d.kind = 1;
                d.nclass = int(c->g.n[v]);
                d.lo = c->g.lo[v];
                d.hv = cell_width(c->g, v);
            } else {
                const int xm = natural_shift_dim(c, m);
                d.kind = 2;
                d.nclass = xm < 0 ? 1 : int(c->g.n[xm]);
                d.field = xm < 0 ? c->d_fields : c->d_fields + field_offset(c, xm);
            }
        }
    }
    if (cudaMemcpyAsync(b->d_kdeg, kd.data(), kd.size() * 4, cudaMemcpyHostToDevice, b->st) != cudaSuccess ||
        cudaMemcpyAsync(b->d_ab, ab.data(), ab.size() * sizeof(BatchAB), cudaMemcpyHostToDevice, b->st) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_tabs, tabs.data(), tabs.size() * sizeof(PolyTab), cudaMemcpyHostToDevice,
                        b->st) != cudaSuccess ||
        cudaMemcpyAsync(b->d_mass_desc, md.data(), md.size() * sizeof(BatchMass), cudaMemcpyHostToDevice,
                        b->st) != cudaSuccess ||
        cudaStreamSynchronize(b->st) != cudaSuccess)
        return cleanup(fail(nullptr, SL_ECUDA, "uploading batch tables"));
    // default shapes (the autotuner's usual picks on 2D x-v batches): whole
    // cells (each problem takes at most its own fibres), two consecutive cells
    // per thread and items of four tiles along dimension 0; one fibre per
    // thread, four cells per walk step and 64-row items along the others
    for (int m = 0; m < b->ndim; ++m) {
        b->tune[m].ft = m == 0 ? kBatchMaxFtUnit : 1;
        b->tune[m].unroll = m == 0 ? 2 : 4;
        b->tune[m].rows = 64;
        b->tune[m].reps = 4;
        sl_status s = rebuild_dim(b, m);
        if (s != SL_OK) {
            fail(nullptr, s, "%s", b->err.c_str());
            return cleanup(s);
        }
    }
    *out = b;
    return SL_OK;
}

void sl_batch_destroy(sl_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->st);
    drop_graph(b);
    if (b->st_tab) {
        cudaStreamSynchronize(b->st_tab);
        cudaStreamDestroy(b->st_tab);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    for (auto& pr : b->ev) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto& it : b->d_items)
        if (it) cudaFree(it);
    if (b->mem) cudaFree(b->mem);
    for (auto* c : b->probs) sl_destroy(c);
    delete b;
}

const char* sl_batch_last_error(const sl_batch* b) { return b ? b->err.c_str() : sl_last_error(nullptr); }

sl_status sl_batch_info(const sl_batch* b, int64_t* cells, int64_t* dof, int64_t* state_bytes)
{
    if (!b || !cells || !dof || !state_bytes) return fail(nullptr, SL_EINVAL, "NULL argument");
    int64_t c = 0, d = 0;
    for (auto* p : b->probs) {
        c += p->cells;
        d += p->cells * p->ncoef;
    }
    *cells = c;
    *dof = d;
    *state_bytes = b->state_bytes;
    return SL_OK;
}

sl_status sl_batch_project(sl_batch* b, int p, int nq, int nterms, const double* weights,
                           const double* params)
{
    sl_status s = check_prob(b, p);
    if (s != SL_OK) return s;
    return forward(b, b->probs[p], sl_project(b->probs[p], nq, nterms, weights, params));
}

sl_status sl_batch_set_coeffs(sl_batch* b, int p, const double* host_aos)
{
    sl_status s = check_prob(b, p);
    if (s != SL_OK) return s;
    return forward(b, b->probs[p], sl_set_coeffs(b->probs[p], host_aos));
}

sl_status sl_batch_get_coeffs(sl_batch* b, int p, double* host_aos)
{
    sl_status s = check_prob(b, p);
    if (s != SL_OK) return s;
    return forward(b, b->probs[p], sl_get_coeffs(b->probs[p], host_aos));
}

sl_status sl_batch_set_fields(sl_batch* b, const double* fields, int64_t count)
{
    if (!b) return fail(nullptr, SL_EINVAL, "batch is NULL");
    int64_t need = 0;
    for (auto* c : b->probs) need += c->nfields;
    if (count != need) return bfail(b, SL_EINVAL, "field count does not match the batch");
    if (need > 0 && !fields) return bfail(b, SL_EINVAL, "fields is NULL");
    int64_t off = 0;
    for (auto* c : b->probs) {
        sl_status s = sl_set_fields(c, fields ? fields + off : nullptr, c->nfields);
        if (s != SL_OK) return forward(b, c, s);
        off += c->nfields;
    }
    return SL_OK;
}

sl_status sl_batch_step(sl_batch* b, sl_splitting sp, double dt, int nsteps)
{
    sl_status s = check_steps(b, sp, dt, nsteps);
    if (s != SL_OK) return s;
    return batch_steps(b, sp, dt, nsteps);
}

sl_status sl_batch_mass(sl_batch* b, double* out)
{
    if (!b || !out) return fail(nullptr, SL_EINVAL, "NULL argument");
    if (b->capturing) return bfail(b, SL_EINVAL, "cannot read the mass during a capture");
    SLB_CUDA(b, launch_batch_mass(b->d_mass_desc, b->nprob, b->parity, b->d_mass, b->st));
    SLB_CUDA(b, cudaMemcpyAsync(out, b->d_mass, size_t(b->nprob) * 8, cudaMemcpyDeviceToHost, b->st));
    SLB_CUDA(b, cudaStreamSynchronize(b->st));
    return SL_OK;
}

sl_status sl_batch_graph_capture(sl_batch* b, sl_splitting sp, double dt, int nsteps)
{
    sl_status s = check_steps(b, sp, dt, nsteps);
    if (s != SL_OK) return s;
    if (!b->st) return bfail(b, SL_EINVAL, "graph capture needs a non-default stream");
    drop_graph(b);
    const int start = b->parity;
    const int sweeps = int(plan_of(b->probs[0], sp).size()) * nsteps;
    const int flip = sweeps & 1;
    for (int gi = 0; gi < (flip ? 2 : 1); ++gi) {
        b->parity = start ^ gi;
        for (auto* c : b->probs) c->cur = b->parity;
        cudaGraph_t graph = nullptr;
        SLB_CUDA(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
        b->capturing = true;
        s = batch_steps(b, sp, dt, nsteps);
        b->capturing = false;
        cudaError_t e = cudaStreamEndCapture(b->st, &graph);
        if (s == SL_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec[gi], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (s != SL_OK || e != cudaSuccess) {
            b->parity = start;
            for (auto* c : b->probs) c->cur = start;
            drop_graph(b);
            return s != SL_OK ? s : bcuda(b, e, "graph capture");
        }
    }
    b->parity = start;
    for (auto* c : b->probs) c->cur = start;
    b->graph_start = start;
    b->graph_flip = flip;
    return SL_OK;
}

sl_status sl_batch_graph_launch(sl_batch* b)
{
    if (!b) return fail(nullptr, SL_EINVAL, "batch is NULL");
    if (b->graph_start < 0) return bfail(b, SL_EINVAL, "no graph captured");
    const int gi = b->parity == b->graph_start ? 0 : 1;
    if (!b->gexec[gi]) return bfail(b, SL_EINVAL, "no graph for the current buffer parity");
    SLB_CUDA(b, cudaGraphLaunch(b->gexec[gi], b->st));
    b->parity ^= b->graph_flip;
    for (auto* c : b->probs) c->cur = b->parity;
    return SL_OK;
}

sl_status sl_batch_synchronize(sl_batch* b)
{
    if (!b) return fail(nullptr, SL_EINVAL, "batch is NULL");
    SLB_CUDA(b, cudaStreamSynchronize(b->st));
    return SL_OK;
}

sl_status sl_batch_autotune(sl_batch* b, int reps)
{
    if (!b) return fail(nullptr, SL_EINVAL, "batch is NULL");
    if (b->capturing) return bfail(b, SL_EINVAL, "cannot autotune during a capture");
    reps = std::max(1, std::min(reps, 50));
    cudaEvent_t e0 = new_event(), e1 = new_event();
    if (!e0 || !e1) return bfail(b, SL_ECUDA, "cudaEventCreate failed");
    sl_status result = SL_OK;
    const bool prof = b->prof;
    b->prof = false;
    for (int m = 0; m < b->ndim && result == SL_OK; ++m) {
        std::vector<sl_batch::Tune> cand;
        if (m == 0) {
            for (int ft = 1; ft <= kBatchMaxFtUnit; ++ft)
                for (int u : {1, 2, 4})
                    if (batch_shape_ok(1, ft, u))
                        for (int r : {1, 4, 8}) cand.push_back({ft, u, 64, r});
        } else {
            for (int ft = 1; ft <= kBatchMaxFtStrided; ++ft)
                for (int u : {2, 4})
                    for (int rows : {32, 64, 128, 1 << 30}) cand.push_back({ft, u, rows, 4});
        }
        // tables of a split substep of 0.05 time units, so that sigma varies
        // between lines as in a real step (they are rebuilt by every sweep)
        cudaError_t e = launch_batch_ab(b->d_ab + size_t(m) * b->nprob, b->d_tabs, b->nprob, b->maxcls[m], 0.05,
                                        b->st);
        if (e != cudaSuccess) {
            result = bcuda(b, e, "batch autotune tables");
            break;
        }
        // time one candidate: a warm-up launch, then reps launches (out of
        // place with the parity restored, so the state is unchanged)
        auto time_one = [&](const sl_batch::Tune& t, float* ms) -> cudaError_t {
            b->tune[m] = t;
            if (rebuild_dim(b, m) != SL_OK) return cudaErrorUnknown;
            const int par = b->parity;
            cudaError_t err = cudaSuccess;
            for (int r = -1; r < reps && err == cudaSuccess; ++r) {
                if (r == 0) err = cudaEventRecord(e0, b->st);
                if (err != cudaSuccess) break;
                const int blocks = b->sms * batch_sweep_occupancy(b->mode, t.ft, t.unroll, m == 0);
                err = launch_batch_sweep(b->mode, t.ft, t.unroll, b->d_args + (size_t(m) * 2 + par) * b->nprob,
                                         b->d_kdeg, b->d_items[m], b->nitems[m], m == 0, t.reps, blocks,
                                         b->d_ctr + m, b->st);
            }
            if (err == cudaSuccess) err = cudaEventRecord(e1, b->st);
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
            result = e == cudaErrorUnknown ? SL_ECUDA : bcuda(b, e, "batch autotune");
            break;
        }
        size_t bi = 0;
        for (size_t q = 1; q < cand.size(); ++q)
            if (t_ms[q] < t_ms[bi]) bi = q;
        const sl_batch::Tune best = cand[bi];
        b->tune[m] = best;
        if (result == SL_OK) result = rebuild_dim(b, m);
    }
    b->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return result;
}

sl_status sl_batch_profile_enable(sl_batch* b, int enable)
{
    if (!b) return fail(nullptr, SL_EINVAL, "batch is NULL");
    b->prof = enable != 0;
    return SL_OK;
}

sl_status sl_batch_profile_query(sl_batch* b, int64_t* launches, double* ms, double* bytes)
{
    if (!b) return fail(nullptr, SL_EINVAL, "batch is NULL");
    SLB_CUDA(b, cudaStreamSynchronize(b->st));
    double tot = 0.0;
    for (int m = 0; m < SL_MAX_DIM; ++m) {
        b->last_dim_launches[m] = 0;
        b->last_dim_ms[m] = 0.0;
    }
    for (size_t q = 0; q < b->ev.size(); ++q) {
        float t = 0.0f;
        SLB_CUDA(b, cudaEventElapsedTime(&t, b->ev[q].first, b->ev[q].second));
        tot += t;
        b->last_dim_launches[b->ev_dim[q]]++;
        b->last_dim_ms[b->ev_dim[q]] += t;
        cudaEventDestroy(b->ev[q].first);
        cudaEventDestroy(b->ev[q].second);
    }
    b->ev.clear();
    b->ev_dim.clear();
    if (launches) *launches = b->prof_launches;
    if (ms) *ms = tot;
    if (bytes) *bytes = 2.0 * double(b->state_bytes) * double(b->prof_launches);
    b->prof_launches = 0;
    return SL_OK;
}

sl_status sl_batch_profile_dims(const sl_batch* b, int64_t* launches, double* ms)
{
    if (!b || !launches || !ms) return fail(nullptr, SL_EINVAL, "NULL argument");
    for (int m = 0; m < SL_MAX_DIM; ++m) {
        launches[m] = b->last_dim_launches[m];
        ms[m] = b->last_dim_ms[m];
    }
    return SL_OK;
}

sl_status sl_batch_set_tune(sl_batch* b, int dim, const sl_tune* t)
{
    if (!b || !t) return fail(nullptr, SL_EINVAL, "NULL argument");
    if (b->capturing) return bfail(b, SL_EINVAL, "cannot change shapes during a capture");
    if (dim < 0 || dim >= b->ndim) return bfail(b, SL_EINVAL, "dim out of range");
    if (t->block != kBatchBlock || t->pipeline != 0 || t->max_blocks_per_sm != 0 || t->reserved != 0)
        return bfail(b, SL_EINVAL, "batches run 128 threads per block, no pipeline and no blocks-per-SM cap");
    if (!batch_shape_ok(dim == 0, t->fibres_per_thread, t->unroll))
        return bfail(b, SL_EINVAL, "(fibres_per_thread, unroll) not provided");
    sl_batch::Tune n = b->tune[dim];
    n.ft = t->fibres_per_thread;
    n.unroll = t->unroll;
    if (dim == 0) {
        const int64_t per = int64_t(kBatchBlock) * t->unroll;
        if (t->chunk < per || t->chunk % per != 0 || t->chunk / per > 8)
            return bfail(b, SL_EINVAL, "chunk along dimension 0 must be 1..8 x 128 x unroll cells");
        n.reps = int(t->chunk / per);
    } else {
        if (t->chunk < 1 || t->chunk > (int64_t(1) << 30)) return bfail(b, SL_EINVAL, "chunk must be >= 1 rows");
        n.rows = int(t->chunk);
    }
    const sl_batch::Tune keep = b->tune[dim];
    b->tune[dim] = n;
    sl_status s = rebuild_dim(b, dim);
    if (s != SL_OK) {
        b->tune[dim] = keep;
        rebuild_dim(b, dim);
    }
    return s;
}

sl_status sl_batch_get_tune(const sl_batch* b, int dim, sl_tune* out)
{
    if (!b || !out) return fail(nullptr, SL_EINVAL, "NULL argument");
    if (dim < 0 || dim >= b->ndim) return fail(nullptr, SL_EINVAL, "dim out of range");
    const auto& t = b->tune[dim];
    out->block = kBatchBlock;
    out->fibres_per_thread = t.ft;
    out->unroll = t.unroll;
    out->pipeline = 0;
    out->chunk = dim == 0 ? int64_t(t.reps) * kBatchBlock * t.unroll : int64_t(t.rows);
    out->max_blocks_per_sm = 0;
    out->reserved = 0;
    return SL_OK;
}

}  // extern "C"
