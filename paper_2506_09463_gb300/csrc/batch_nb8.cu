// batch_nb8.cu -- the batched kernels with panels of 8 reflectors (a
// setting of the batch autotuner, see batch.cu), compiled apart so that the
// settings build in parallel.
#include "batch_core.cuh"

namespace slqr {

BatchKernels batch_kernels_nb8(int tc) {
  switch (tc) {
    case 32: return batch_kernels_of<8, 32>();
    case 64: return batch_kernels_of<8, 64>();
    default: return BatchKernels{};
  }
}

}  // namespace slqr
