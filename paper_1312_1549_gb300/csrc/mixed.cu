// Mixed-precision line searches (tensor-core contractions with float64 state).
#include "omm_mixed.cuh"

#include <stdexcept>

namespace omm {

struct MixedState {
  int m, n;
};

MixedState* mixed_create(cudaStream_t, int, int, const double*, const double*) {
  throw CudaError{cudaErrorNotSupported, "mixed precision is not built in this version"};
}
void mixed_update_H(MixedState*, cudaStream_t, const double*) {}
void mixed_destroy(MixedState* ms) { delete ms; }
void mixed_iterate(MixedState*, cudaStream_t, Scalars*, double*, double*, double*, double*, double*,
                   double*, double*, double*, double*, double*, const double*, const double*, bool) {}

}  // namespace omm
