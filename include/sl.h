/*
 * sl.h -- C ABI of the GB300 (sm_103a) semi-Lagrangian discontinuous Galerkin
 * projection-sweep library (libsl.so).
 *
 * Method: L. Einkemmer, "A mixed precision semi-Lagrangian algorithm and its
 * performance on accelerators", HPCS 2016 (arXiv:1603.07008).
 *
 *   - Sec. II: time splitting reduces the Vlasov equation to a sequence of
 *     one-dimensional constant-coefficient advections, eq. (advection),
 *     u_t + a u_x = 0, whose exact solution is a translation.
 *   - Sec. II-A: on every cell the solution is a polynomial of degree p
 *     (o = p+1 coefficients) in the Legendre basis, coefficients by eq. (cj).
 *     Translating and projecting back gives the update rule
 *         c_i^{n+1} = A c_{i*}^n + B c_{i*+1}^n
 *     with o x o matrices A, B that depend only on the time step.
 *   - Sec. II-A, III-A: c_0 carries the mass, so keeping c_0 in FP64 and the
 *     other coefficients in lower precision conserves mass to double precision.
 *
 * Conventions of this library (readings of the paper):
 *   - shift in cells s = a*tau/h = sigma + alpha, sigma = floor(s), alpha in
 *     [0,1); source cells of cell i are i-sigma (matrix A) and i-sigma-1
 *     (matrix B); every dimension is periodic.
 *   - d dimensions (1..6) with a tensor-product Legendre basis, o^d
 *     coefficients per cell, multi-index J = sum_m j_m o^m (j_0 fastest);
 *     cells in row-major order with dimension 0 fastest.  A sweep along
 *     dimension m applies the 1D update to every fibre of coefficients that
 *     varies only in j_m; the shift is constant along each line and may
 *     depend on one orthogonal cell coordinate (shift_dim).
 *   - Vlasov-type splitting: x-dimension m is paired with v-dimension
 *     pair[m].  The x-sweep along m moves with the cell-centre velocity of
 *     its v-cell, the v-sweep along pair[m] with the field E_m sampled at the
 *     x_m cell centres.
 *
 * Storage modes (the "split coefficient store"):
 *   SL_FP64      every coefficient in FP64 (the paper's "# double = o").
 *   SL_MIX_FP32  cell mean c_{0..0} in an FP64 plane, all other coefficients
 *                in FP32 planes ("# double = 1"); mean row computed in FP64.
 *   SL_MIX_BF16, SL_MIX_FP16
 *                mean in FP64, the others in BF16 / FP16 scaled per cell by a
 *                power of two stored in an FP32 plane; arithmetic in FP32.
 *                (Not in the paper: a further compression step of the same
 *                idea.)  Requires o^d <= 128.
 *   SL_FP32, SL_MIX_FP32_D2, SL_MIX_FP32_D3
 *                the paper's other "# double" columns: 0, 2 and 3 coefficients
 *                per dimension in FP64 (see sl_storage below).
 *
 * Memory: sl_create allocates the device state (two copies, ping-pong) with
 * cudaMalloc and owns it; sl_destroy frees it.  Host arrays passed in are
 * owned by the caller and only read (or written) during the call.  All device
 * work is ordered on the CUDA stream given to sl_create (NULL = legacy
 * default stream).  Calls that return results to the host (sl_mass,
 * sl_get_coeffs, sl_get_cells, sl_batch_mass, sl_batch_get_coeffs,
 * sl_profile_query) synchronise that stream; the others only enqueue work.
 * A context must not be used from two host threads at once.
 *
 * Errors: every call returns an sl_status; nothing is thrown across the ABI.
 * On failure sl_last_error(ctx) (or sl_last_error(NULL) when no context
 * exists yet) returns a message.  Invalid arguments are rejected before any
 * device work is enqueued, so the state is unchanged.
 */
#ifndef SL_H
#define SL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SL_MAX_DIM 6
#define SL_MAX_DEGREE 3

typedef enum {
    SL_OK = 0,
    SL_EINVAL = -1,    /* invalid argument (grid, degree, dimension, size, non-finite value) */
    SL_ENOMEM = -2,    /* device or host allocation failed */
    SL_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
    SL_ETIMEOUT = -4,  /* reserved for a bounded device-side wait; no kernel of this library spins on a flag */
    SL_ENAN = -5,      /* non-finite value in an input array */
    SL_ENOTSUP = -6    /* valid request this library does not support (e.g. scaled mode with o^d > 128) */
} sl_status;

/* Storage of the Legendre coefficients c_{j_0..j_{d-1}} of a cell (Sec. III-A,
 * "# double" = how many coefficients per dimension are kept in FP64):
 *   SL_FP64         every coefficient in FP64 (# double = o)
 *   SL_MIX_FP32     the cell mean c_{0..0} in FP64, the others in FP32 (# double = 1)
 *   SL_MIX_BF16/16  the cell mean in FP64, the others BF16 / FP16 times a
 *                   per-cell FP32 power-of-two scale
 *   SL_FP32         every coefficient in FP32, FP32 arithmetic (# double = 0;
 *                   mass is conserved only to FP32 rounding, Table II)
 *   SL_MIX_FP32_D2  the coefficients whose every index j_m < 2 in FP64, the
 *                   others in FP32 (# double = 2; in 1D c_0, c_1); degree >= 2
 *   SL_MIX_FP32_D3  every index j_m < 3 in FP64 (# double = 3); degree 3
 * In the stores of # double = q >= 1 the rows of FP64 coefficients are computed
 * in FP64, the others in FP32. */
typedef enum {
    SL_FP64 = 0,
    SL_MIX_FP32 = 1,
    SL_MIX_BF16 = 2,
    SL_MIX_FP16 = 3,
    SL_FP32 = 4,
    SL_MIX_FP32_D2 = 5,
    SL_MIX_FP32_D3 = 6
} sl_storage;

typedef enum {
    SL_LIE = 0,     /* x-dims with dt, then v-dims with dt */
    SL_STRANG = 1   /* x-dims with dt/2, v-dims with dt, x-dims with dt/2 */
} sl_splitting;

/* Periodic box [lo_m, hi_m) with n_m cells per dimension, m < ndim.
 * pair[m] >= 0: x-dimension m is advected with the velocity coordinate
 * pair[m]; pair[m] = -1 otherwise.  Unused entries are ignored. */
typedef struct {
    int32_t ndim;
    int64_t n[SL_MAX_DIM];
    double lo[SL_MAX_DIM];
    double hi[SL_MAX_DIM];
    int32_t pair[SL_MAX_DIM];
} sl_grid;

typedef struct sl_ctx sl_ctx;

/* Sizes of a context's state (one copy of the ping-pong pair). */
typedef struct {
    int64_t cells;          /* prod n_m */
    int64_t ncoef;          /* o^d */
    int64_t dof;            /* cells * ncoef */
    int64_t plane_stride;   /* elements between consecutive coefficient planes */
    int64_t state_bytes;    /* algorithmic bytes of one state: cells * (8 + (o^d-1) * elem [+ 4 scale]),
                               cells * (8 n_lo + 4 n_hi) for the split stores (sl_plane_layout) */
    int64_t alloc_bytes;    /* device bytes allocated by the context (both copies + tables) */
    int32_t degree;
    int32_t storage;        /* sl_storage */
    int32_t record_slots;   /* 0: planar store (coefficient J >= 1 in plane J-1, planes
                               plane_stride apart); R > 0: the scaled store keeps the
                               higher coefficients of every cell in one record of R
                               16-bit slots, slot J holding coefficient J (slot 0 and
                               slots >= o^d are zero), chosen for 6D/5D with degree 1
                               and 3D with degree 3 */
} sl_info;

/* ---------------------------------------------------------------- setup */

/* Create a context for `grid`, polynomial degree `degree` (0..3, o = degree+1
 * Legendre coefficients per dimension, Sec. II-A) and storage mode `storage`.
 * `cuda_stream` is a cudaStream_t (may be NULL).  Allocates two copies of the
 * state on the current device.  The state starts at zero.
 * Errors: SL_EINVAL (ndim not in 1..6, n_m < 1, hi_m <= lo_m, degree out of
 * range, bad pair), SL_ENOTSUP (scaled mode with o^d > 128), SL_ENOMEM,
 * SL_ECUDA. */
sl_status sl_create(const sl_grid* grid, int degree, sl_storage storage, void* cuda_stream,
                    sl_ctx** out);

/* Layout of one copy of the state for (grid, degree, storage): plane_stride
 * (elements between coefficient planes, cells rounded up to 64),
 * record_slots (0: planar), and the bytes of its three arrays: the FP64 mean
 * plane [plane_stride], the higher coefficients ([o^d - 1][plane_stride]
 * planes, or [cells][record_slots] records, in the storage's element type)
 * and the FP32 scale plane [plane_stride] (0 bytes for the unscaled stores).
 * The stores of # double = 0, 2, 3 (SL_FP32, SL_MIX_FP32_D2, SL_MIX_FP32_D3)
 * have n_lo = q^d FP64 planes [n_lo][plane_stride] in place of the mean plane
 * (none for SL_FP32) and n_hi = o^d - q^d FP32 planes, both in increasing
 * coefficient order J = sum_m j_m o^m (the FP64 plane of the cell mean first).
 * Errors as sl_create's argument checks. */
typedef struct {
    int64_t plane_stride;
    int32_t record_slots;
    int32_t reserved;
    int64_t mean_bytes;
    int64_t hi_bytes;
    int64_t scale_bytes;
} sl_layout;
sl_status sl_plane_layout(const sl_grid* grid, int degree, sl_storage storage, sl_layout* out);

/* As sl_create, but the two copies of the state live in caller-owned device
 * memory (e.g. framework tensors): planes = {mean_0, hi_0, scale_0, mean_1,
 * hi_1, scale_1}, each 256-byte aligned and of the sizes sl_plane_layout
 * gives (the scale pointers may be NULL for the unscaled stores).  The
 * context neither initialises nor frees them; the caller keeps them alive
 * until sl_destroy.  Which copy holds the current state changes with every
 * sweep (sl_get_planes reads the current one).  Errors: as sl_create, and
 * SL_EINVAL for a NULL or misaligned plane pointer. */
sl_status sl_create_external(const sl_grid* grid, int degree, sl_storage storage, void* cuda_stream,
                             void* const* planes, sl_ctx** out);

/* Canaries, the sanitizer of this library (no GPU fault is ever provoked):
 * every array of a context's allocation is followed by a guard band of at
 * least 256 bytes, and the padding of every owned plane past the last cell
 * (up to plane_stride) is filled too, all with the byte 0xA5 at creation.  No
 * kernel or copy of the library writes there.  *corrupted_bytes = the number
 * of those bytes that no longer hold 0xA5 (0 for a sound run).  Synchronises.
 * The planes of sl_create_external are the caller's and are not covered.
 * Errors: SL_EINVAL (NULL, or during a capture), SL_ECUDA. */
sl_status sl_check_guards(sl_ctx* ctx, int64_t* corrupted_bytes);
/* Test hooks of the failure paths (host side only, no device fault):
 * sl_debug_fail_alloc(n), n >= 1: the n-th device or pinned-host allocation
 * the library makes from now on fails as if out of memory (later ones succeed
 * again); n = 0 switches the hook off.  Process-wide.  SL_EINVAL for n < 0.
 * sl_debug_corrupt_guard: overwrites the first byte of the context's first
 * guard band (inside its own allocation), so that a test can see
 * sl_check_guards report it. */
sl_status sl_debug_fail_alloc(int64_t n);
sl_status sl_debug_corrupt_guard(sl_ctx* ctx);

/* Free the context and its device memory (after synchronising its stream).
 * NULL is ignored. */
void sl_destroy(sl_ctx* ctx);

/* Last error message of `ctx`, or of the calling thread's last failed
 * sl_create / sl_batch_create when ctx is NULL.  Never NULL. */
const char* sl_last_error(const sl_ctx* ctx);

/* Fill *out with the context's sizes.  Host only. */
sl_status sl_get_info(const sl_ctx* ctx, sl_info* out);

/* Bytes of one state (the algorithmic byte model) without creating a
 * context: cells * (8 + (o^d - 1) * elem (+ 4 for the per-cell scale)),
 * elem = 8 / 4 / 2 / 2 for SL_FP64 / SL_MIX_FP32 / SL_MIX_BF16 / SL_MIX_FP16,
 * and cells * (8 n_lo + 4 n_hi) for the stores of # double = q (see
 * sl_plane_layout).
 * Sec. III-A gives the memory reduction this model implies (1.6x for
 * 1D order 4 with c_0 in FP64).  Host only. */
sl_status sl_state_bytes(const sl_grid* grid, int degree, sl_storage storage, int64_t* bytes);

/* Evaluate the update matrices A(alpha), B(alpha) of Sec. II-A (update rule)
 * on the host from the exact polynomial-in-alpha tables the device kernels
 * use.  A, B: row-major o x o FP64, caller-owned.  alpha in [0,1).
 * Host only (no device work). */
sl_status sl_ab_host(int degree, double alpha, double* A, double* B);

/* ---------------------------------------------------------------- data */

/* Upload coefficients: host_aos is [cells][o^d] FP64 (layout above),
 * caller-owned.  The library splits them into the mean plane and the
 * low-precision planes (round to nearest even; per-cell power-of-two scale in
 * the scaled modes).  Errors: SL_EINVAL (NULL), SL_ENAN (non-finite input,
 * state unchanged), SL_ECUDA. */
sl_status sl_set_coeffs(sl_ctx* ctx, const double* host_aos);

/* Download all coefficients, decoded to FP64, into host_aos [cells][o^d].
 * Synchronises. */
sl_status sl_get_coeffs(sl_ctx* ctx, double* host_aos);

/* Download the coefficients of `ncells` cells (flat indices, each in
 * [0, cells)) into host_out [ncells][o^d].  Synchronises. */
sl_status sl_get_cells(sl_ctx* ctx, const int64_t* cells, int64_t ncells, double* host_out);

/* Raw planes in the store's own layout (for checkpoints and for callers that
 * keep the state on the host between steps):
 *   mean  [cells]            FP64 cell means c_{0..0} ([n_lo][cells] FP64
 *                            planes for SL_MIX_FP32_D2/D3; unused, may be NULL,
 *                            for SL_FP32; hi is then [n_hi][cells] FP32,
 *                            see sl_plane_layout)
 *   hi    [o^d - 1][cells]   coefficient J >= 1 at hi[(J-1)*cells + cell], in
 *                            the store's element type (FP64, FP32, or the
 *                            BF16 / FP16 bit patterns); with cell records
 *                            (sl_info.record_slots = R > 0) hi is [cells][R]
 *                            and coefficient J is hi[cell*R + J]
 *   scale [cells]            FP32 per-cell scales (scaled modes; NULL otherwise)
 * sl_set_planes enqueues the host-to-device copies on the context's stream
 * and returns; the host arrays must stay valid and unchanged until the stream
 * has passed them (sl_synchronize).  Pinned host memory makes the copies
 * asynchronous.  Values are copied verbatim, without validation.
 * sl_get_planes copies the current state out and synchronises. */
sl_status sl_set_planes(sl_ctx* ctx, const double* mean, const void* hi, const float* scale);
sl_status sl_get_planes(sl_ctx* ctx, double* mean, void* hi, float* scale);

/* Project an initial condition onto the cells, eq. (cj), on the device:
 *   u0(x) = sum_t weights[t] prod_m g_{t,m}(x_m),
 *   g(x)  = exp(-gamma (x - mu)^2) cos(kappa x + phi),
 * params[(t*ndim + m)*4 + {0,1,2,3}] = {gamma, mu, kappa, phi}.  Each
 * dimension uses an nq-point Gauss-Legendre rule (1 <= nq <= 32).  The
 * tensor-product rule on a product factorises, so the cost is one 1D
 * projection per factor and cell coordinate.  Host arrays, caller-owned. */
sl_status sl_project(sl_ctx* ctx, int nq, int nterms, const double* weights,
                     const double* params);

/* ---------------------------------------------------------------- the sweep */

/* One sweep along `dim`: every cell gets A(alpha) c[i-sigma] + B(alpha)
 * c[i-sigma-1] (Sec. II-A, update rule) along that dimension.
 * shift_dim = -1: one shift for all lines, nshift = 1.
 * shift_dim = q != dim: shifts[i] applies to the lines whose coordinate along
 * q is i, nshift = n[q].  Shifts are in cells (a * tau / h_dim), host array,
 * caller-owned.  Matrices are built on the device for every shift class.
 * Errors: SL_EINVAL (dim / shift_dim / nshift), SL_ENAN (non-finite shift). */
sl_status sl_advect(sl_ctx* ctx, int dim, int shift_dim, const double* shifts, int64_t nshift);

/* Electric fields for the v-sweeps: for every x-dimension m (pair[m] >= 0) in
 * increasing m, n[m] samples of E_m at the x_m cell centres, concatenated.
 * count must equal the sum of those n[m].  Copied to the device. */
sl_status sl_set_fields(sl_ctx* ctx, const double* fields, int64_t count);

/* nsteps split time steps of size dt (Sec. II, splitting): Lie or Strang
 * over the x/v pairs of the grid.  x-sweep along m: shift v_j tau / h_m with
 * v_j the cell centre of v-dimension pair[m]; v-sweep along pair[m]: shift
 * E_m(x_i) tau / h_{pair[m]}.  Needs sl_set_fields when the grid has pairs.
 * Enqueues only.  Each step builds every dimension's A/B table once (the
 * v-dimensions' on a stream of the context's own, forked from and joined
 * back to the context's stream within the step), so all of a step's work is
 * ordered on the context's stream as seen from outside. */
sl_status sl_step(sl_ctx* ctx, sl_splitting splitting, double dt, int nsteps);

/* Mass M = (prod_m h_m) sum_i c_{i;0..0} (Sec. II-A: c_0 is the cell mean),
 * reduced in FP64 with a fixed-shape tree (run-to-run deterministic).
 * Synchronises. */
sl_status sl_mass(sl_ctx* ctx, double* out);

/* Allocation-free mass reduction.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library call cudaMalloc -- for
 * example a host application that owns all device memory through its own
 * pool or arena, or a latency-critical loop where a cudaMalloc (which may
 * synchronise the device) is not allowed.  It computes
 *     *d_out = cell_volume * sum_{i < cells} d_mean[i]
 * with the same fixed-shape FP64 reduction as sl_mass, but its scratch (the
 * per-block partial sums) is a fixed 8 KB __device__ array inside the
 * library (1024 FP64 slots), which every GPU that loads the library keeps
 * until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   d_mean       device pointer, `cells` FP64 values (caller-owned)
 *   cells        1 .. 2^31 - 1; anything else returns SL_EINVAL
 *   cell_volume  product of the cell widths (SL_ENAN if NaN)
 *   d_out        device pointer to one FP64 result (caller-owned)
 *   cuda_stream  cudaStream_t the work is enqueued on (NULL = legacy default)
 * Enqueues only; the result is valid once the stream reaches it.  The first
 * call on a device looks up the scratch array's device address on that device
 * (the current one), so make that first call before any stream capture.  The
 * address is kept for the life of the process and belongs to the device's
 * primary context (the one the CUDA runtime uses): do not call this entry
 * point under another context made current through the driver API, nor after
 * cudaDeviceReset on that device (the kept address then names freed memory).
 * All calls share the one scratch array: calls whose work overlaps on the GPU
 * (different streams, no ordering between them) race and may return wrong
 * sums.  Each call rewrites every scratch slot it reads, so a previous call's
 * leftovers never leak into a result.  Errors: SL_EINVAL (NULL pointer or
 * cells out of range), SL_ENAN, SL_ECUDA (address lookup or launch failed).
 * sl_last_error does not cover this call. */
sl_status sl_mass_noalloc(const double* d_mean, int64_t cells, double cell_volume, double* d_out,
                          void* cuda_stream);

/* Self-test of the device-side binary32 <-> binary64 conversions the mean
 * row of the low-precision stores uses (integer-pipe forms of the IEEE 754
 * conversions).  For host arrays of n elements (1 <= n <= 2^26):
 * f_out[2i] = fl32(d_in[i]) and f_out[2i+1] = fl32(-d_in[i]), rounded to
 * nearest with ties to even (f_out holds 2n floats); d_out[i] = f_in[i]
 * (exact).  Exception, the binary32 subnormal range: results of magnitude
 * below 2^-126 become a signed zero, and subnormal f_in map to doubles of
 * magnitude below 2^-126.  *mismatches = the number of elements on which the
 * library's branching and branch-free forms of these conversions disagree
 * (must be 0).  Synchronous, on the default stream.  Errors: SL_EINVAL,
 * SL_ENOMEM, SL_ECUDA; sl_last_error does not cover this call. */
sl_status sl_selftest_conversions(const double* d_in, const float* f_in, int64_t n, float* f_out,
                                  double* d_out, int64_t* mismatches);
/* Self-test of the device-side difference of two widened binary32 values the
 * mean row uses: out[i] = (double)a[i] - (double)b[i], formed on the integer
 * pipe when exact (both normal, exponents at most 28 apart) and by the FP64
 * subtraction otherwise (binary32 subnormal inputs as in sl_selftest_conversions).
 * *mismatches = elements on which the integer form and the FP64 subtraction
 * disagree (must be 0).  Host arrays of n elements (1 <= n <= 2^26).
 * Synchronous, on the default stream.  Errors: SL_EINVAL, SL_ENOMEM, SL_ECUDA. */
sl_status sl_selftest_sub_widened(const float* a, const float* b, int64_t n, double* out, int64_t* mismatches);
/* Measured FP64 arithmetic rate of the current device, the roofline of the
 * FP64 store (its sweep costs 2o FP64 FMAs per coefficient against the
 * 4o - 1 flops per coefficient of Sec. II-A, at the device's FP64 rate):
 * 8 independent chains of FP64 FMAs with register operands per thread, the
 * better of 4 and 8 resident blocks of 256 threads per multiprocessor, each
 * timed with CUDA events on `cuda_stream` after a shorter warm-up launch;
 * every chain runs about `iters` FMAs.  *flops_per_s = 2 * FMAs / seconds.
 * 1 <= iters <= 2^24 (2^14 takes about 65 ms per shape on GB300).
 * Allocates 24 bytes of device memory for the duration of the call;
 * synchronous.  Errors: SL_EINVAL, SL_ENOMEM, SL_ECUDA. */
sl_status sl_selftest_fp64_rate(int64_t iters, void* cuda_stream, double* flops_per_s);

/* Self-consistent field (NEXT to the sweep: the Vlasov-Poisson system of
 * Sec. II in 1+1 dimensions).  For a grid with one x dimension paired with
 * one v dimension, enable = 1 makes sl_step and sl_graph_capture compute the
 * field of the v-sweep from the state before every v-sweep, instead of
 * taking the samples of sl_set_fields: d_x E = rho - rho_bar with
 * rho_i = h_v sum_j c_{i,j;0} (the x-cell average of int f dv) and rho_bar
 * its mean, E at the x-cell centres = sum_{j<i} q_j + q_i / 2 with
 * q = (rho - rho_bar) h_x, minus its mean (int E dx = 0).  Allocates a
 * scratch of (ceil(n_v / 256) + 1) n_x + 1 doubles on first use (not during
 * a capture).  Errors: SL_EINVAL (other grids), SL_ENOMEM. */
sl_status sl_set_poisson(sl_ctx* ctx, int enable);
/* The field of the current state at the x-cell centres (host array of n_x
 * doubles), and the field energy (1/2) sum_i E_i^2 h_x.  Synchronise. */
sl_status sl_get_field(sl_ctx* ctx, double* field);
sl_status sl_field_energy(sl_ctx* ctx, double* energy);

/* Nodal-in-velocity x-sweeps (NEXT to the sweep: in several dimensions the
 * velocity of the x-advection v d_x f varies inside a v-cell).  enable = 1
 * makes sl_step and sl_graph_capture sweep every x-dimension m with the
 * velocity taken at the o Gauss-Legendre nodes eta_q of each cell of its v-
 * dimension p = pair[m], instead of at the cell centre:
 *   U_q(l)    = sum_jv c_{l,jv} P_jv(eta_q)                  (values at node q)
 *   U'_q      = the update rule of Sec. II-A for U_q with the shift
 *               (lo_p + (j + 1/2 + eta_q / 2) h_p) tau / h_m, j the v-cell
 *   c'_{jx,jv} = (2 jv + 1) / 2 sum_q w_q P_jv(eta_q) U'_q(jx)  (eq. (cj) along v)
 * for every fibre of coefficients varying in (j_m, j_p).  The mean stays
 * conserved to FP64 rounding in the mixed store.  Stores SL_FP64 and
 * SL_MIX_FP32 (SL_ENOTSUP otherwise).  Allocates the node velocities and
 * tables on first use (not during a capture).  Errors: SL_EINVAL (no x-
 * dimension with a pair), SL_ENOTSUP, SL_ENOMEM. */
sl_status sl_set_nodal_velocity(sl_ctx* ctx, int enable);
/* One nodal-in-velocity x-sweep along the x-dimension dim over time tau
 * (shifts v tau / h_dim at the nodes, as above).  Errors: SL_EINVAL (dim not an
 * x-dimension), SL_ENAN (tau not finite), as sl_set_nodal_velocity. */
sl_status sl_advect_nodal(sl_ctx* ctx, int dim, double tau);

/* Arithmetic of the sweeps of the stores with FP32 planes (Sec. III-A and
 * Table II state which coefficients a store keeps in double precision, not
 * the precision the update rule of Sec. II-A is evaluated in).
 *   SL_ARITH_STORE (default): the rows of FP32 coefficients are computed in
 *     FP32 arithmetic (the FP64 rows as the store's own sweeps describe);
 *     the launch shapes of sl_set_tune / sl_autotune apply.
 *   SL_ARITH_FP64: every row is computed in FP64 from the stored values
 *     widened to FP64 with the FP64 matrices, and the new FP32 coefficients
 *     are rounded once (to nearest, ties to even) on store; the store keeps
 *     its layout and bytes.  Then a sweep differs from the FP64 store's only
 *     by the rounding of what the store holds.  One launch shape (one fibre
 *     per thread), bound by the FP64 pipe like the FP64 store.
 * Takes effect for the sweeps issued after the call (a graph captured before
 * keeps its kernels).  Stores SL_MIX_FP32, SL_FP32, SL_MIX_FP32_D2,
 * SL_MIX_FP32_D3; for SL_FP64 both values are accepted and change nothing.
 * Errors: SL_EINVAL (unknown value, NULL ctx, during a capture), SL_ENOTSUP
 * (SL_ARITH_FP64 with the scaled stores or with nodal-in-velocity x-sweeps
 * enabled; sl_set_nodal_velocity and sl_advect_nodal in turn return
 * SL_ENOTSUP while SL_ARITH_FP64 is set). */
typedef enum { SL_ARITH_STORE = 0, SL_ARITH_FP64 = 1 } sl_arith;
sl_status sl_set_arithmetic(sl_ctx* ctx, int arith);

/* Capture nsteps of sl_step into a CUDA graph (replacing a previous one) and
 * replay it with sl_graph_launch.  Fields must be set before capture.  Every
 * replay builds its shift tables from the context's field array as it is
 * then, so fields set later with sl_set_fields (ordered on the context's
 * stream) are used from the next replay on. */
sl_status sl_graph_capture(sl_ctx* ctx, sl_splitting splitting, double dt, int nsteps);
sl_status sl_graph_launch(sl_ctx* ctx);
/* Capture nsteps sweeps of sl_advect(ctx, dim, shift_dim, shifts, nshift),
 * each with its table build, into a CUDA graph (replacing a previous graph)
 * that sl_graph_launch replays.  The graph keeps its own device copy of the
 * shifts.  Same argument checks as sl_advect; nsteps >= 1.  A 1D context of
 * the FP64 store with one shift (shift_dim = -1) whose line fits one
 * thread-block cluster's shared memory (about 8000 cells at degree 2) runs
 * the nsteps sweeps, each building its matrices, in one kernel launch; the
 * results are the same bits as nsteps sl_advect calls. */
sl_status sl_graph_capture_advect(sl_ctx* ctx, int dim, int shift_dim, const double* shifts, int64_t nshift,
                                  int nsteps);

/* Wait for all work of the context's stream. */
sl_status sl_synchronize(sl_ctx* ctx);

/* ---------------------------------------------------------------- batches */

/* Many independent problems advanced together (the sweeps are independent
 * per problem, Sec. II-A; nothing is exchanged between problems).  Every
 * split substep is one table launch over all problems and one persistent
 * sweep launch over a work list of equal-sized tiles of all problems, so
 * problems of very different sizes share the GPU evenly.
 * All problems must have the same ndim and the same pair[] (the same split
 * structure); extents, box and degree may differ.  Degrees 0..2; stores
 * SL_FP64 and SL_MIX_FP32 (SL_ENOTSUP otherwise).  The batch owns one
 * single-problem state per problem; every call below except the per-problem
 * set/get/project is one launch (or one synchronisation) for the whole batch.
 * Errors as for the single-problem calls; sl_batch_last_error gives the
 * message (sl_last_error(NULL) for a failed sl_batch_create). */
typedef struct sl_batch sl_batch;

sl_status sl_batch_create(int nprob, const sl_grid* grids, const int* degrees, sl_storage storage,
                          void* cuda_stream, sl_batch** out);
void sl_batch_destroy(sl_batch* batch);
const char* sl_batch_last_error(const sl_batch* batch);
/* Totals over all problems: cells, degrees of freedom, bytes of one state. */
sl_status sl_batch_info(const sl_batch* batch, int64_t* cells, int64_t* dof, int64_t* state_bytes);
/* Per-problem data, as sl_project / sl_set_coeffs / sl_get_coeffs. */
sl_status sl_batch_project(sl_batch* batch, int prob, int nq, int nterms, const double* weights,
                           const double* params);
sl_status sl_batch_set_coeffs(sl_batch* batch, int prob, const double* host_aos);
sl_status sl_batch_get_coeffs(sl_batch* batch, int prob, double* host_aos);
/* Fields of every problem, concatenated in problem order (each as for
 * sl_set_fields). */
sl_status sl_batch_set_fields(sl_batch* batch, const double* fields, int64_t count);
/* nsteps Lie or Strang steps of size dt for every problem (as sl_step). */
sl_status sl_batch_step(sl_batch* batch, sl_splitting splitting, double dt, int nsteps);
/* Mass of every problem into out[nprob]; synchronises. */
sl_status sl_batch_mass(sl_batch* batch, double* out);
/* As sl_graph_capture / sl_graph_launch for the batch: each replay builds the
 * problems' tables from their fields as they are then (sl_batch_set_fields
 * between replays is used by the next one). */
sl_status sl_batch_graph_capture(sl_batch* batch, sl_splitting splitting, double dt, int nsteps);
sl_status sl_batch_graph_launch(sl_batch* batch);
sl_status sl_batch_synchronize(sl_batch* batch);
/* Time the provided work-list shapes (fibres per thread, cells per walk step,
 * chunks per line) for every dimension and keep the fastest. */
sl_status sl_batch_autotune(sl_batch* batch, int reps);
/* As sl_profile_enable / sl_profile_query, over the batched sweep launches;
 * bytes = 2 x (sum of the problems' state bytes) per launch. */
sl_status sl_batch_profile_enable(sl_batch* batch, int enable);
sl_status sl_batch_profile_query(sl_batch* batch, int64_t* launches, double* ms, double* bytes);
/* Per sweep dimension m (launches[SL_MAX_DIM], ms[SL_MAX_DIM]): the launches
 * and milliseconds of the last sl_batch_profile_query's window. */
sl_status sl_batch_profile_dims(const sl_batch* batch, int64_t* launches, double* ms);


/* ---------------------------------------------------------------- launch shapes */

/* Launch shape of the sweep kernel along one dimension.
 *   block              threads per block (multiple of 32; <= 256 for dimension 0,
 *                      <= 128 otherwise)
 *   fibres_per_thread  coefficient fibres one thread updates: 1, 2, 3, 4 or 9
 *                      along dimension 0; 1, 2 or 3 otherwise.  The scaled
 *                      stores need a cell-wide maximum: a thread takes every
 *                      fibre of its cell (o^(d-1)) or a share of them, with
 *                      the maximum exchanged in shared memory; the shares
 *                      provided are 16, 8, 4 of 32 and 8, 4 of 16 fibres
 *                      (k = 1), 9, 3 of 27 and 3 of 9 (k = 2), 4 of 16 (k = 3).
 *   unroll             along dimensions > 0: cells per walk step, 1, 2 or 4
 *                      (4 only with 1 or 2 fibres per thread); along
 *                      dimension 0: cells per thread, 1, or 16 / element size
 *                      (4 for FP32, 2 for FP64) for the 16-byte vector form,
 *                      which needs n_0 divisible by it and 1..4 fibres per
 *                      thread (FP64 and FP32 stores)
 *   chunk              cells one thread walks along dimensions > 0 (1..n_dim)
 *   Cell records (sl_info.record_slots = R > 0) take one of two forms:
 *     one thread per cell: fibres_per_thread = o^(d-1), block <= 128,
 *       unroll 1 (plain) or 2 (prefetching walk); along dimension 0 chunk 0
 *       means one thread per target cell, chunk > 0 a walk;
 *     lane groups (degree 1 in 5 or 6 dimensions): fibres_per_thread = 8,
 *       G = R/16 lanes share a cell, each holding 16 slots; every dimension,
 *       dimension 0 included, is walked (chunk >= 1), unroll 1, 2 or 4 cells
 *       per walk step, block <= 256.
 *   max_blocks_per_sm  0, or 4, 5 or 6: the register walk along dimensions > 0
 *                      (FP64 and FP32 stores, pipeline 0) runs at most that
 *                      many blocks per SM (fewer concurrent walks can use the
 *                      DRAM pages better; the autotuner measures it)
 *   pipeline           0: the walk keeps the previous cell in registers;
 *                      4 or 8: the walk streams its source rows through a
 *                      per-thread cp.async ring of that many rows in shared
 *                      memory (FP64 and FP32 stores, dimensions > 0, with 1 or
 *                      2 fibres per thread, or 3 with pipeline 4; unroll
 *                      is ignored)
 *   The stores of # double = 2, 3 (SL_MIX_FP32_D2/D3) take fibres_per_thread 1,
 *   unroll 1 along dimension 0 and 1 or 2 elsewhere, block <= 256 / 128, no
 *   pipeline and no block limit; SL_FP32 takes every shape of SL_MIX_FP32.
 * Every shape computes the same result; only the speed differs. */
typedef struct {
    int32_t block;
    int32_t fibres_per_thread;
    int32_t unroll;
    int32_t pipeline;
    int64_t chunk;
    int32_t max_blocks_per_sm;
    int32_t reserved;   /* must be 0 */
} sl_tune;

sl_status sl_get_tune(const sl_ctx* ctx, int dim, sl_tune* out);
/* Errors: SL_EINVAL for a shape this library does not provide. */
sl_status sl_set_tune(sl_ctx* ctx, int dim, const sl_tune* tune);

/* Autotuner: for every dimension, time each provided launch shape `reps`
 * times on the current state (out of place, so the state is unchanged) and
 * keep the fastest.  Synchronises.  Must not be called during a capture. */
sl_status sl_autotune(sl_ctx* ctx, int reps);

/* The batch's work-list shape along dimension dim: block = threads per
 * block, fibres_per_thread = the most fibres per thread (each problem takes
 * at most its own), unroll = cells per walk step, chunk = rows per work item
 * (dim > 0) or cells per work item (dim 0); pipeline is 0. */
sl_status sl_batch_get_tune(const sl_batch* batch, int dim, sl_tune* out);
/* Set the batch's work-list shape along dimension dim, in the terms of
 * sl_batch_get_tune: block must be 128 and pipeline and max_blocks_per_sm
 * 0; dimension 0 takes fibres_per_thread 1..3 with unroll (cells per thread)
 * 1 or 2, or 1..2 with 4, and chunk a multiple of 128 x unroll up to
 * 8 x 128 x unroll cells per item; the other dimensions take
 * fibres_per_thread 1..2, unroll 1, 2 or 4 and chunk >= 1 rows per item.
 * Errors: SL_EINVAL for a shape this library does not provide. */
sl_status sl_batch_set_tune(sl_batch* batch, int dim, const sl_tune* tune);

/* ---------------------------------------------------------------- profiling */

/* When enabled, every sweep-kernel launch is bracketed by CUDA events on the
 * context's stream.  sl_profile_query synchronises and returns, since the
 * last reset, the number of sweep launches, their summed device time (ms) and
 * their summed algorithmic bytes (read + write of every state coefficient
 * once), then resets the counters.  Off by default. */
sl_status sl_profile_enable(sl_ctx* ctx, int enable);
sl_status sl_profile_query(sl_ctx* ctx, int64_t* launches, double* ms, double* bytes);

/* The per-dimension split of the last sl_profile_query: launches[m] and ms[m]
 * for every sweep dimension m < ndim (caller arrays of SL_MAX_DIM entries).
 * Host only. */
sl_status sl_profile_dims(const sl_ctx* ctx, int64_t* launches, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* SL_H */
