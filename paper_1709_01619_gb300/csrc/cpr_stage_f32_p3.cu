// Stage kernel instantiation: float, p = 3.
#include "cpr_stage_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_STAGE(float, 3)
}
