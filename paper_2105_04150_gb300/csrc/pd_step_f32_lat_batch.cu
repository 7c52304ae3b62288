// Batch build of the regular-lattice FP32 step kernel (see PD_LAT_BATCH in
// pd_step_f32_lat.cu): the instances of a batch of lattice models in one launch.
#define PD_LAT_BATCH 1
#include "pd_step_f32_lat.cu"
