// step_mode_plain.cu -- the plain variant of the persistent step kernel
// (step_kernel.cuh), for every launch shape.  One translation unit per
// variant, so that they compile in parallel.
#include "step_kernel.cuh"

namespace snn {
template const void* step_fn_mode<0>(int, bool);
}  // namespace snn
