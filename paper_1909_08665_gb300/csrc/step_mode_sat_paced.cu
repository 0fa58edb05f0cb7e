// step_mode_sat_paced.cu -- the wrap-counting variant, paced to wall-clock
// time of the persistent step kernel (step_kernel.cuh), for every launch
// shape.  One translation unit per variant, so that they compile in parallel.
#include "step_kernel.cuh"

namespace snn {
template const void* step_fn_mode<kModeSat | kModePaced>(int, bool);
}  // namespace snn
