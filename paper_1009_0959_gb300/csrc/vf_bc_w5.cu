// Class kernels of the batched form, 5 x 5 windows (vf_batch_class.cuh).
#include "vf_batch_class.cuh"

namespace vf {
cudaError_t launch_class_w5(int crit, int apx, const BatchImage* imgs, const int* begin, int count,
                            unsigned int* counter, int tiles, cudaStream_t s) {
  return launch_class_window<5>(crit, apx, imgs, begin, count, counter, tiles, s);
}
}  // namespace vf
