// step_mode_paced.cu -- the variant paced to wall-clock time
// (snn_set_realtime) of the persistent step kernel (step_kernel.cuh), for
// every launch shape.  One translation unit per variant, so that they compile
// in parallel.
#include "step_kernel.cuh"

namespace snn {
template const void* step_fn_mode<kModePaced>(int, bool);
}  // namespace snn
