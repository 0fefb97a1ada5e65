// Wide line kernels (wf_wide.cuh): the layout check and the FP32 instantiation.
#include "wf_wide.cuh"

namespace wf {

bool wide_supported(const Geom& g) {
  return g.tp >= 1 && g.tp <= wide::kWideCta && g.n >= 1 && g.n <= NMAX && g.lpl >= 1 && g.lpl <= 32 &&
         g.tp == g.n * g.lpl;
}

template void launch_line_wide<float>(const LineArgs<float>&, int, cudaStream_t);
template void launch_line_wide_multi<float>(const std::vector<LineArgs<float>>&, int, cudaStream_t);

}  // namespace wf
