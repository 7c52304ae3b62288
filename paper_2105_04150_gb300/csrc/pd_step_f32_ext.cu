// Extended-epilogue build of the FP32 step kernel: velocity-Verlet, the smooth
// loading start and the read-only force pass (see PD_F32_EXT in pd_step_f32.cu),
// so the plain Euler-Cromer build carries none of their cost.
#define PD_F32_EXT 1
#include "pd_step_f32.cu"
