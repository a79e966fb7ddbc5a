// sl_sweep_f32all.cu -- sweep kernels of the all-FP32 store ("# double" = 0).
#define SL_FP_MODE M_F32ALL
#define SL_FP_LAUNCHER launch_sweep_f32all
#include "sl_sweep_fp.inc"
