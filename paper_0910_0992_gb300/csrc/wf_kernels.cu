// Line kernels of the temporal preconditioner and the Wilson matrix M.
//
// k_line is the kernel behind every C_L / C_R / T^-1 / T^-dag application and every
// fused "hop + time-line solve" step of the Schur operator (§II.A, §II.B):
//   source   : the site's own spinor (SRC_LOAD) or D_s of the other parity (SRC_HOP)
//   pre-axpy : v <- xpre + apre v
//   solves   : per spin half, copy / T^-dag (forward) / T^-1 (backward) / skip
//   post-axpy: out <- xpost + apost v, optionally with the two halves exchanged,
//              optionally accumulating |out|^2 per right-hand side
// One warp handles 32 / lpl time lines; lpl lanes share a line, n sites each. The three
// kernels of the Schur operator are compiled with their source and solve ops fixed, so
// each carries only its own code; every other use goes through one kernel that selects
// them at run time.
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <type_traits>
#include <vector>

#include "wf_internal.h"
#include "wf_line.cuh"
#include "wf_line_kernels.cuh"

namespace wf {

// In the axial frame the FP32 hop kernels of the Schur operator (K-b, K-c) run as the
// one-thread-per-site kernels of wf_wide.cu: measured on GB300 (24^3 x 128) 1.15-1.3x faster
// than k_line. The scan-heavy, memory-light K-a stays on k_line, which amortises the scan over
// n sites per lane; FP64 arithmetic stays on k_line too. Environment WF_WIDE=0 disables the
// wide FP32 kernels, WF_WIDE=2 uses them for every FP32 axial line operation.
static bool use_wide(const Geom& g, int kind, bool fp32) {
  static const int mode = []() {  // read once (thread-safe initialisation)
    const char* e = std::getenv("WF_WIDE");
    return (e && e[0] == '0') ? 0 : (e && e[0] == '2') ? 2 : 1;
  }();
  if (!mode || !wide_supported(g)) return false;
  return mode == 2 || (fp32 && (kind == LK_SCHUR_B || kind == LK_SCHUR_C));
}

template <typename R>
static void launch_line_impl(const LineArgs<R>& a, int kind, bool axial, cudaStream_t s) {
  if (a.h16) {
    // FP16 spinor storage (FP32 arithmetic): K-a on this kernel, the hop kernels on the wide one
    if constexpr (std::is_same<R, float>::value) {
      if (axial && kind == LK_SCHUR_A && a.g.n >= 1 && a.g.n <= NMAX) {
        k_line<float, true, SRC_LOAD, OP_FWD, OP_SKIP, true><<<line_blocks(a), kLineThreads, 0, s>>>(a);
        WF_CUDA(cudaGetLastError());
        return;
      }
      if (axial && (kind == LK_SCHUR_B || kind == LK_SCHUR_C) && wide_supported(a.g)) {
        launch_line_wide(a, kind, s);
        return;
      }
    }
    throw Error(1, "line kernel: FP16 storage only for the Schur operator's kernels in the axial frame");
  }
  if constexpr (sizeof(R) == 4) {
    const bool wide = a.variant == 1 ? wide_supported(a.g) : a.variant == 2 ? false : use_wide(a.g, kind, true);
    if (axial && wide) {
      launch_line_wide(a, kind, s);
      return;
    }
  }
  if (a.g.n < 1 || a.g.n > NMAX_LONG) throw Error(1, "unsupported sites per lane");
  const int b = line_blocks(a);
  if (a.g.n > NMAX) {  // lines longer than 128 slots: the long-line variant (wf_kernels_long_*.cu)
    launch_line_long<R>(a, kind, axial, s);
    return;
  }
#define WF_KL(AXV, SRCV, OPUV, OPLV) k_line<R, AXV, SRCV, OPUV, OPLV><<<b, kLineThreads, 0, s>>>(a)
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

// the same arguments for the double-float kernels: FP64 arrays are read and written as such
// (Cx<df64> has the size and alignment of Cx<double>), scalars are split on the host
template <typename A, typename B>
static const Cx<A>* as_cx(const Cx<B>* p) { return reinterpret_cast<const Cx<A>*>(p); }
static LineArgs<df64> line_args_df(const LineArgs<double>& a) {
  LineArgs<df64> b;
  std::memset(&b, 0, sizeof(b));  // every field defined, including ones added later
  b.g = a.g;
  b.parity = a.parity;
  b.nrhs = a.nrhs;
  b.opu = a.opu;
  b.opl = a.opl;
  b.src = a.src;
  b.src_up = as_cx<df64>(a.src_up);
  b.src_lo = as_cx<df64>(a.src_lo);
  b.ut = as_cx<df64>(a.ut);
  b.pl = as_cx<df64>(a.pl);
  b.us_out = as_cx<df64>(a.us_out);
  b.us_nbr = as_cx<df64>(a.us_nbr);
  b.lamb = as_cx<df64>(a.lamb);
  b.lamf = as_cx<df64>(a.lamf);
  b.xpre = as_cx<df64>(a.xpre);
  b.apre = df64(a.apre);
  b.xpost = as_cx<df64>(a.xpost);
  b.apost = df64(a.apost);
  b.swap_out = a.swap_out;
  b.stream_out = a.stream_out;
  b.out = reinterpret_cast<Cx<df64>*>(a.out);
  b.norm2 = a.norm2;
  b.inv_mu = df64(a.inv_mu);
  b.bc = df64(a.bc);
  b.drop_job = -1;
  b.df = 0;
  b.order = a.order;
  b.nbr = a.nbr;
  b.active = a.active;
  return b;
}

template <typename R>
void launch_line(const LineArgs<R>& a, int kind, bool axial, cudaStream_t s) {
  if constexpr (std::is_same<R, double>::value) {
    // double-float runs one site per thread (with n sites per lane the double-width state of
    // k_line spills); the caller's-gauge frame stays in FP64
    if (a.df && axial && wide_supported(a.g)) {
      launch_line_wide(line_args_df(a), kind, s);
      return;
    }
  }
  launch_line_impl<R>(a, kind, axial, s);
}
// K-a, K-b or K-c (LK_SCHUR_A/B/C, axial frame) on this kernel over a ragged batch of lattices, in
// launches of up to kMaxLattices lattices
template <typename R>
void launch_line_multi(const std::vector<LineArgs<R>>& as, int kind, cudaStream_t s) {
  if (kind != LK_SCHUR_A && kind != LK_SCHUR_B && kind != LK_SCHUR_C)
    throw Error(1, "multi-lattice line kernel: K-a, K-b or K-c");
  for (size_t first = 0; first < as.size(); first += kMaxLattices) {
    MultiLineArgs<R> M;
    std::memset(&M, 0, sizeof(M));
    M.n = (int)std::min<size_t>(kMaxLattices, as.size() - first);
    int blocks = 0;
    for (int k = 0; k < M.n; ++k) {
      const LineArgs<R>& a = as[first + k];
      if (a.g.n < 1 || a.g.n > NMAX || a.h16) throw Error(1, "multi-lattice line kernel: unsupported layout");
      M.a[k] = a;
      M.blk0[k] = blocks;
      blocks += line_blocks(a);
    }
    M.blk0[M.n] = blocks;
    if (blocks == 0) continue;
    if (kind == LK_SCHUR_A)
      k_line_multi<R, true, SRC_LOAD, OP_FWD, OP_SKIP><<<blocks, kLineThreads, 0, s>>>(M);
    else if (kind == LK_SCHUR_B)
      k_line_multi<R, true, SRC_HOP, OP_FWD, OP_BWD><<<blocks, kLineThreads, 0, s>>>(M);
    else
      k_line_multi<R, true, SRC_HOP, OP_COPY, OP_BWD><<<blocks, kLineThreads, 0, s>>>(M);
    WF_CUDA(cudaGetLastError());
  }
}
template void launch_line_multi<float>(const std::vector<LineArgs<float>>&, int, cudaStream_t);

template void launch_line<float>(const LineArgs<float>&, int, bool, cudaStream_t);
template void launch_line<double>(const LineArgs<double>&, int, bool, cudaStream_t);

template <typename R>
void launch_apply_M(const MArgs<R>& a, bool axial, cudaStream_t s) {
  if (a.g.n < 1 || a.g.n > NMAX_LONG) throw Error(1, "unsupported sites per lane");
  const int lines = a.nrhs * a.g.Nl;
  const int warps = (lines + a.g.lpw - 1) / a.g.lpw;
  const int blocks = (warps * 32 + kLineThreads - 1) / kLineThreads;
  if (a.g.n > NMAX) {  // lines longer than 128 slots (wf_kernels_long_*.cu)
    launch_apply_M_long<R>(a, axial, s);
    return;
  }
  if (axial)
    k_apply_M<R, true, NMAX><<<blocks, kLineThreads, 0, s>>>(a);
  else
    k_apply_M<R, false, NMAX><<<blocks, kLineThreads, 0, s>>>(a);
  WF_CUDA(cudaGetLastError());
}
template void launch_apply_M<float>(const MArgs<float>&, bool, cudaStream_t);
template void launch_apply_M<double>(const MArgs<double>&, bool, cudaStream_t);

}  // namespace wf
