// Velocity-Verlet build of the double-word step kernel (see pd_step_dw.cu).
#define PD_DW_VV 1
#include "pd_step_dw.cu"
