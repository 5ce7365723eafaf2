// Element-wise passes and order dispatch: float state.
#include "cpr_aux_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_AUX(float)
}
