// Bilinear-softening build of the FP32 step kernel: the same source with the
// per-slot bond integrity compiled in (see PD_F32_SOFT in pd_step_f32.cu), so
// the plain PMB kernel carries none of its cost.
#define PD_F32_SOFT 1
#include "pd_step_f32.cu"
