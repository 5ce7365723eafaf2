// Stage kernel instantiation: float, p = 2.
#include "cpr_stage_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_STAGE(float, 2)
}
