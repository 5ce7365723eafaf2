// Batched stage kernel instantiation: float, tile family 1.
#include "cpr_batch_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_BATCH(float, 1)
}
