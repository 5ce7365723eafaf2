// Stage kernel instantiation: float, p = 4.
#include "cpr_stage_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_STAGE(float, 4)
}
