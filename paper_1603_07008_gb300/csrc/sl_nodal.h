// sl_nodal.h -- arguments of the nodal-in-velocity x-sweep (sl_nodal.cu).
// Not part of the public ABI (include/sl.h is).
#pragma once

#include "sl_internal.cuh"

namespace sl {

// Floats per v-cell of the FP32 node record (NodalArgs::na32) and the place of
// its alpha_bar (after the o values alpha_q, in the first 16 bytes when o <= 3).
constexpr int kNa32 = 8;
__host__ __device__ constexpr int na32_abar(int o) { return o < 4 ? 3 : 4; }

// One nodal x-sweep along xdim (paired with vdim) from src to dst.  tab holds
// the classes j * o + q (v-cell j, node q).  The node tables are filled by
// nodal_setup.
struct NodalArgs {
    Planes src, dst;
    ShiftTable tab;
    uint32_t cells;
    uint32_t N, NV;            // extents of the x- and v-dimensions
    uint32_t inner_x;          // cells between neighbours along x
    FastDiv fdInnerX, fdNX;    // cell -> x coordinate: (cell / inner_x) % N
    FastDiv fdInnerV, fdNV;    // cell -> v-cell:       (cell / inner_v) % NV
    int64_t pstride;
    int ostride, vstride;      // o^xdim, o^vdim
    int ndim, xdim, vdim, O;
    uint32_t nfib2;            // fibres varying in (j_x, j_v): o^(ndim - 2)
    int off32;                 // 1: plane_stride * o^ndim < 2^31 (32-bit element offsets)
    uint32_t nrunx, nruns;     // runs of consecutive x-cells (set by the launcher): per x-line, in all
    FastDiv fdRunX;            // run -> run along its x-line: (run / inner_x) % nrunx
    double eval64[kMaxO][kMaxO];   // P_jv(eta_q) at [q][jv]
    double back64[kMaxO][kMaxO];   // (2 jv + 1) / 2 w_q P_jv(eta_q) at [jv][q]; row 0 = wmean
    double wmean[kMaxO];           // w_q / 2 rounded to sum to exactly 1
    float wmean32[kMaxO];          // the same in FP32
    const double* abar;            // per v-cell: alpha_bar = sum_q wmean[q] alpha_q (launch_nodal_abar)
    const float* na32;             // per v-cell, kNa32 floats: alpha_q rounded to FP32, then at
                                   // na32_abar(o) the FP32 fma chain sum_q wmean32[q] alpha32_q
    float eval32[kMaxO][kMaxO];
    float back32[kMaxO][kMaxO];
};

// Gauss-Legendre nodes eta[o] (ascending) and weights[o] of degree K's o = K + 1
// points, and the node tables of a.
void nodal_setup(int K, double* eta, double* weights, NodalArgs* a);
// One nodal x-sweep over every cell and every one of the nfib2 = o^(d-2)
// fibres of coefficients varying in (j_x, j_v); the launcher picks the grid
// (per target, or runs of targets along x-dimensions > 0 in the mixed store)
// and fills the run fields of its copy of a.
cudaError_t launch_sweep_nodal(int K, int mode, const NodalArgs& a, int nfib2, cudaStream_t st);
// alpha_bar of every v-cell j < nv from the node table's alpha[j * o + q]:
// the fma chain sum_q wmean[q] alpha_q from 0, in node order, and the FP32
// record na32[j * kNa32 ..] (alpha_q rounded to nearest FP32, then the FP32
// chain of wmean32[q] and those values); the mean's fibre of the mixed store
// reads them instead of forming them per target.
cudaError_t launch_nodal_abar(const double* alpha, int nv, int o, const double* wmean, const float* wmean32,
                              double* abar, float* na32, cudaStream_t st);

}  // namespace sl
