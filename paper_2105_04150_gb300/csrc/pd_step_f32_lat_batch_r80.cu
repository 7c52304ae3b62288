// Batch build of the regular-lattice FP32 step kernel allocated for 3 resident
// blocks of 256 threads per SM (80 registers): the compiled variant of
// pd_step_f32_lat_batch.cu that pd_autotune times against it.
#define PD_LAT_BATCH 1
#define PD_LAT_MIN_BLOCKS 3
#include "pd_step_f32_lat.cu"
