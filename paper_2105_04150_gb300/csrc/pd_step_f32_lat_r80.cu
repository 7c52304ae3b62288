// The regular-lattice FP32 step kernel allocated for 3 resident blocks of 256
// threads per SM (80 registers) instead of 4 (64): a compiled variant that
// pd_autotune times against the default (see PD_LAT_MIN_BLOCKS in
// pd_step_f32_lat.cu).
#define PD_LAT_MIN_BLOCKS 3
#include "pd_step_f32_lat.cu"
