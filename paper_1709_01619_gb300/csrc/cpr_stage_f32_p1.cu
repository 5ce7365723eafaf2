// Stage kernel instantiation: float, p = 1.
#include "cpr_stage_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_STAGE(float, 1)
}
