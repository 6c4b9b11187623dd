// Class kernels of the batched form, 7 x 7 windows (vf_batch_class.cuh).
#include "vf_batch_class.cuh"

namespace vf {
cudaError_t launch_class_w7(int crit, int apx, const BatchImage* imgs, const int* begin, int count,
                            unsigned int* counter, int tiles, cudaStream_t s) {
  return launch_class_window<7>(crit, apx, imgs, begin, count, counter, tiles, s);
}
}  // namespace vf
