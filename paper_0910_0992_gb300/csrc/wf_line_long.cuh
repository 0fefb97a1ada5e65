// Launchers of the line kernels' long-line variant (time lines of 129 to 256 sites: up to
// NMAX_LONG sites per lane), instantiated per precision in wf_kernels_long_f32.cu and
// wf_kernels_long_f64.cu; launch_line and launch_apply_M (wf_kernels.cu) hand such lattices here.
#pragma once

#include "wf_line_kernels.cuh"

namespace wf {

template <typename R>
void launch_line_long(const LineArgs<R>& a, int kind, bool axial, cudaStream_t s) {
  if (a.g.n <= NMAX || a.g.n > NMAX_LONG || a.h16) throw Error(1, "long-line kernel: unsupported line layout");
  const int b = line_blocks(a);
#define WF_KL(AXV, SRCV, OPUV, OPLV) k_line<R, AXV, SRCV, OPUV, OPLV, false, NMAX_LONG><<<b, kLineThreads, 0, s>>>(a)
  if (axial) {
    switch (kind) {
      case LK_SCHUR_A: WF_KL(true, SRC_LOAD, OP_FWD, OP_SKIP); break;
      case LK_SCHUR_B: WF_KL(true, SRC_HOP, OP_FWD, OP_BWD); break;
      case LK_SCHUR_C: WF_KL(true, SRC_HOP, OP_COPY, OP_BWD); break;
      default: WF_KL(true, -1, -1, -1); break;
    }
  } else {
    switch (kind) {
      case LK_SCHUR_A: WF_KL(false, SRC_LOAD, OP_FWD, OP_SKIP); break;
      case LK_SCHUR_B: WF_KL(false, SRC_HOP, OP_FWD, OP_BWD); break;
      case LK_SCHUR_C: WF_KL(false, SRC_HOP, OP_COPY, OP_BWD); break;
      default: WF_KL(false, -1, -1, -1); break;
    }
  }
#undef WF_KL
  WF_CUDA(cudaGetLastError());
}

template <typename R>
void launch_apply_M_long(const MArgs<R>& a, bool axial, cudaStream_t s) {
  if (a.g.n <= NMAX || a.g.n > NMAX_LONG) throw Error(1, "long-line kernel: unsupported line layout");
  const int lines = a.nrhs * a.g.Nl;
  const int warps = (lines + a.g.lpw - 1) / a.g.lpw;
  const int blocks = (warps * 32 + kLineThreads - 1) / kLineThreads;
  if (axial)
    k_apply_M<R, true, NMAX_LONG><<<blocks, kLineThreads, 0, s>>>(a);
  else
    k_apply_M<R, false, NMAX_LONG><<<blocks, kLineThreads, 0, s>>>(a);
  WF_CUDA(cudaGetLastError());
}

}  // namespace wf
