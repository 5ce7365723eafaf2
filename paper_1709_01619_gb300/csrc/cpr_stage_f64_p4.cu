// Stage kernel instantiation: double, p = 4.
#include "cpr_stage_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_STAGE(double, 4)
}
