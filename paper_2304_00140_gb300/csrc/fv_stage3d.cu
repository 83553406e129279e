// fv_stage3d.cu -- 3D double instantiations of the stage kernel.
#define FV_ND 3
#define FV_REAL double
#define FV_IS_FLOAT 0
#define FV_SUFFIX 3d
#include "fv_stage_inst.cuh"
