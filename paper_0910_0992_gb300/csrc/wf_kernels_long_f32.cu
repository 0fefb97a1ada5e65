// The line kernels' long-line variant (time lines of 129 to 256 sites), float precision.
#include "wf_line_long.cuh"

namespace wf {
template void launch_line_long<float>(const LineArgs<float>&, int, bool, cudaStream_t);
template void launch_apply_M_long<float>(const MArgs<float>&, bool, cudaStream_t);
}  // namespace wf
