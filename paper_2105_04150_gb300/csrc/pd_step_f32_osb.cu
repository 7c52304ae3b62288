// State-based build of the FP32 kernels: the ordinary state-based model's
// dilation and force kernels over the bond-based step's records and helpers
// (see PD_F32_OSB in pd_step_f32.cu).
#define PD_F32_OSB 1
#include "pd_step_f32.cu"
