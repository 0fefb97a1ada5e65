// Wide line kernels (wf_wide.cuh), double-float instantiation: the FP64 steps of FP32-iteration
// solves (reliable updates, source preparation, reconstruction).
#include "wf_wide.cuh"

namespace wf {

template void launch_line_wide<df64>(const LineArgs<df64>&, int, cudaStream_t);

}  // namespace wf
