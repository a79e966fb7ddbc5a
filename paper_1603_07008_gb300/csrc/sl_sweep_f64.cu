// sl_sweep_f64.cu -- sweep kernels of the all-FP64 store.
#define SL_FP_MODE M_FP64
#define SL_FP_LAUNCHER launch_sweep_f64
#include "sl_sweep_fp.inc"
