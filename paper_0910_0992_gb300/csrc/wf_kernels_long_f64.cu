// The line kernels' long-line variant (time lines of 129 to 256 sites), double precision.
#include "wf_line_long.cuh"

namespace wf {
template void launch_line_long<double>(const LineArgs<double>&, int, bool, cudaStream_t);
template void launch_apply_M_long<double>(const MArgs<double>&, bool, cudaStream_t);
}  // namespace wf
