// Batched stage kernel instantiation: double, tile family 1.
#include "cpr_batch_inst.cuh"
namespace cpr {
CPR_INSTANTIATE_BATCH(double, 1)
}
