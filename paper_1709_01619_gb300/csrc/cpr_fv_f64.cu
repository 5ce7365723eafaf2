// FV stage kernel, double.
#include "cpr_fv_inst.cuh"

CPR_INSTANTIATE_FV(double)
