// Element-wise passes and order dispatch: double state.
#include "cpr_aux_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_AUX(double)
}
