// Tensor-core (tcgen05) cell products -- placeholder until the kernel lands.
#include "common.cuh"

namespace pawfe {

void tc_prepare(paw_context *, paw_precision, cudaStream_t) {
  throw Error{PAW_ERR_UNSUPPORTED, "tensor-core cell kernels are not built yet"};
}

void cell_apply_tc(paw_context *, paw_precision, const float *, int, float *, int, int, float, cudaStream_t) {
  throw Error{PAW_ERR_UNSUPPORTED, "tensor-core cell kernels are not built yet"};
}

}  // namespace pawfe
