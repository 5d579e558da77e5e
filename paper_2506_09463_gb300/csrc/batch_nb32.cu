// batch_nb32.cu -- the batched kernels with panels of 32 reflectors (a
// setting of the batch autotuner, see batch.cu), compiled apart so that the
// settings build in parallel.
#include "batch_core.cuh"

namespace slqr {

BatchKernels batch_kernels_nb32(int tc) {
  switch (tc) {
    case 16: return batch_kernels_of<32, 16>();
    case 32: return batch_kernels_of<32, 32>();
    case 64: return batch_kernels_of<32, 64>();
    default: return BatchKernels{};
  }
}

}  // namespace slqr
