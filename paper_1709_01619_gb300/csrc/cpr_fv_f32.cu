// FV stage kernel, float.
#include "cpr_fv_inst.cuh"

CPR_INSTANTIATE_FV(float)
