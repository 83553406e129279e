// fv_stage3f.cu -- 3D float instantiations of the stage kernel.
#define FV_ND 3
#define FV_REAL float
#define FV_IS_FLOAT 1
#define FV_SUFFIX 3f
#include "fv_stage_inst.cuh"
