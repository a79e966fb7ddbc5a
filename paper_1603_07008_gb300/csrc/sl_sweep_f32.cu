// sl_sweep_f32.cu -- sweep kernels of the mixed FP64-mean / FP32 store.
#define SL_FP_MODE M_F32
#define SL_FP_LAUNCHER launch_sweep_f32
#include "sl_sweep_fp.inc"
