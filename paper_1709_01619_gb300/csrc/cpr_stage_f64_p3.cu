// Stage kernel instantiation: double, p = 3.
#include "cpr_stage_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_STAGE(double, 3)
}
