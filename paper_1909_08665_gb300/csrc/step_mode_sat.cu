// step_mode_sat.cu -- the variant for networks whose input of one step can
// leave the int32 range: it counts the wrap-arounds of every ring cell and
// raises the saturation status of the persistent step kernel
// (step_kernel.cuh), for every launch shape.  One translation unit per
// variant, so that they compile in parallel.
#include "step_kernel.cuh"

namespace snn {
template const void* step_fn_mode<kModeSat>(int, bool);
}  // namespace snn
