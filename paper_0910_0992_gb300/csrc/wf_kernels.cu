// Line kernels of the temporal preconditioner and the Wilson matrix M.
//
// k_line is the one kernel behind every C_L / C_R / T^-1 / T^-dag application and
// every fused "hop + time-line solve" step of the Schur operator (§II.A, §II.B):
//   source   : the site's own spinor (SRC_LOAD) or D_s of the other parity (SRC_HOP)
//   pre-axpy : v <- xpre + apre v
//   solves   : per spin half, copy / T^-dag (forward) / T^-1 (backward) / skip
//   post-axpy: out <- xpost + apost v, optionally with the two halves exchanged
// One warp handles 32 / lpl time lines; lpl lanes share a line, n sites each.
#include "wf_internal.h"
#include "wf_line.cuh"

namespace wf {

constexpr int kLineThreads = 128;

template <typename R, int N, bool FWD>
__device__ __forceinline__ void solve_half(Vec3<R> (&v)[N][4], int s0, const Cx<R>* ut_line, const Cx<R>* lam,
                                           const Geom& g, int jj, R inv_mu, R bc) {
  constexpr int NS = sizeof(R) == 4 ? 2 : 1;
#pragma unroll
  for (int sp = 0; sp < 2; sp += NS) {
    Vec3<R> w[N][NS];
#pragma unroll
    for (int m = 0; m < N; ++m)
#pragma unroll
      for (int s = 0; s < NS; ++s) w[m][s] = v[m][s0 + sp + s];
    tline_solve<R, N, NS, FWD>(w, ut_line, lam, g, jj, inv_mu, bc);
#pragma unroll
    for (int m = 0; m < N; ++m)
#pragma unroll
      for (int s = 0; s < NS; ++s) v[m][s0 + sp + s] = w[m][s];
  }
}

template <typename R, int N, int SRC>
__global__ void __launch_bounds__(kLineThreads) k_line(const LineArgs<R> A) {
  const Geom& g = A.g;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lg_raw = warp * g.lpw + lane / g.lpl;
  const bool active = lg_raw < A.nrhs * g.Nl;
  const int lg = active ? lg_raw : 0;  // idle lanes still join the warp shuffles
  const int rhs = lg / g.Nl, l = lg - rhs * g.Nl;
  const int jj = lane % g.lpl;
  const int tp = g.tp;
  const size_t base = (size_t)lg * NSPIN_C * tp;

  Vec3<R> v[N][4];
  if (SRC == SRC_HOP) {
    hop_spatial<R, N>(v, A, rhs, l, jj);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const int sl = m * g.lpl + jj;
      v[m][0] = ldvec(A.src_up + base, tp, sl);
      v[m][1] = ldvec(A.src_up + base + 3 * tp, tp, sl);
      v[m][2] = ldvec(A.src_lo + base, tp, sl);
      v[m][3] = ldvec(A.src_lo + base + 3 * tp, tp, sl);
    }
  }
  if (A.xpre) {
#pragma unroll
    for (int m = 0; m < N; ++m)
#pragma unroll
      for (int s = 0; s < 4; ++s) v[m][s] = vaxpy(A.apre, v[m][s], ldvec(A.xpre + base + 3 * s * tp, tp, m * g.lpl + jj));
  }

  const Cx<R>* ut_line = A.ut + (size_t)l * NLINK_C * tp;
  if (A.opu == OP_FWD)
    solve_half<R, N, true>(v, 0, ut_line, A.lamf + (size_t)l * 9, g, jj, A.inv_mu, A.bc);
  else if (A.opu == OP_BWD)
    solve_half<R, N, false>(v, 0, ut_line, A.lamb + (size_t)l * 9, g, jj, A.inv_mu, A.bc);
  if (A.opl == OP_FWD)
    solve_half<R, N, true>(v, 2, ut_line, A.lamf + (size_t)l * 9, g, jj, A.inv_mu, A.bc);
  else if (A.opl == OP_BWD)
    solve_half<R, N, false>(v, 2, ut_line, A.lamb + (size_t)l * 9, g, jj, A.inv_mu, A.bc);

  if (!active) return;
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const int sl = m * g.lpl + jj;
    const bool valid = jj * N + m < g.T;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int op = h ? A.opl : A.opu;
      if (op == OP_SKIP) continue;
      const int dh = A.swap_out ? 1 - h : h;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int comp0 = dh * 6 + s * 3;
        Vec3<R> val = valid ? v[m][2 * h + s] : vzero<R>();
        if (A.xpost) val = vaxpy(A.apost, val, ldvec(A.xpost + base + comp0 * tp, tp, sl));
        stvec(A.out + base + comp0 * tp, tp, sl, val);
      }
    }
  }
}

template <typename R>
void launch_line(const LineArgs<R>& a, int src, cudaStream_t s) {
  const int lines = a.nrhs * a.g.Nl;
  const int warps = (lines + a.g.lpw - 1) / a.g.lpw;
  const int blocks = (warps * 32 + kLineThreads - 1) / kLineThreads;
#define WF_LINE_CASE(NN)                                                          \
  case NN:                                                                        \
    if (src == SRC_HOP)                                                           \
      k_line<R, NN, SRC_HOP><<<blocks, kLineThreads, 0, s>>>(a);                  \
    else                                                                          \
      k_line<R, NN, SRC_LOAD><<<blocks, kLineThreads, 0, s>>>(a);                 \
    break;
  switch (a.g.n) {
    WF_LINE_CASE(1)
    WF_LINE_CASE(2)
    WF_LINE_CASE(3)
    WF_LINE_CASE(4)
    default:
      throw Error(1, "unsupported sites per lane");
  }
#undef WF_LINE_CASE
  WF_CUDA(cudaGetLastError());
}
template void launch_line<float>(const LineArgs<float>&, int, cudaStream_t);
template void launch_line<double>(const LineArgs<double>&, int, cudaStream_t);

// ----------------------------------------------------------------------------
// Wilson matrix M = mu - D_t - D_s / gamma_f (§II, Eq. for M) on the output parity:
// out_p = mu psi_p - D_t psi_p - D_s psi_q / gamma_f   (or x + a * that).
// Dirac-Pauli basis: P_- = (1 - gamma_t)/2 keeps spins 2-3, P_+ spins 0-1, so
// D_t psi(t) = P_- U_t(t) psi(t+1) + P_+ U_t^dag(t-1) psi(t-1), sign bc across the wrap.
// ----------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(kLineThreads) k_apply_M(const MArgs<R> A) {
  const Geom& g = A.g;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lg = warp * g.lpw + lane / g.lpl;
  if (lg >= A.nrhs * g.Nl) return;
  const int rhs = lg / g.Nl, l = lg - rhs * g.Nl;
  const int jj = lane % g.lpl;
  const int tp = g.tp, T = g.T;
  const size_t base = (size_t)lg * NSPIN_C * tp;

  // spatial hop from the other parity
  LineArgs<R> H;
  H.g = g;
  H.parity = A.parity;
  H.src_up = A.psi_q;
  H.src_lo = A.psi_q + 6 * tp;
  H.us_out = A.us_out;
  H.us_nbr = A.us_nbr;
  Vec3<R> h[N][4];
  hop_spatial<R, N>(h, H, rhs, l, jj);

  const Cx<R>* ut_line = A.ut + (size_t)l * NLINK_C * tp;
  const Cx<R>* pp = A.psi_p + base;
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const int t = jj * N + m;
    const int sl = m * g.lpl + jj;
    Vec3<R> res[4];
    if (t < T) {
      const int tf = t == T - 1 ? 0 : t + 1;
      const int tb = t == 0 ? T - 1 : t - 1;
      const R sf = t == T - 1 ? A.bc : R(1);
      const R sb = t == 0 ? A.bc : R(1);
      const int slf = slot_of(g, tf), slb = slot_of(g, tb);
      const Mat3<R> Uf = ldmat(ut_line, tp, sl);
      const Mat3<R> Ub = ldmat(ut_line, tp, slb);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        Vec3<R> dt = s < 2 ? matvec_dag(Ub, ldvec(pp + 3 * s * tp, tp, slb)) : matvec(Uf, ldvec(pp + 3 * s * tp, tp, slf));
        const R sg = s < 2 ? sb : sf;
        Vec3<R> r = vscale(A.mu, ldvec(pp + 3 * s * tp, tp, sl));
        r = vaxpy(-sg, dt, r);
        res[s] = vaxpy(-A.inv_gf, h[m][s], r);
      }
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s) res[s] = vzero<R>();
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      Vec3<R> val = res[s];
      if (A.x) val = vaxpy(A.a, val, ldvec(A.x + base + 3 * s * tp, tp, sl));
      stvec(A.out + base + 3 * s * tp, tp, sl, val);
    }
  }
}

template <typename R>
void launch_apply_M(const MArgs<R>& a, cudaStream_t s) {
  const int lines = a.nrhs * a.g.Nl;
  const int warps = (lines + a.g.lpw - 1) / a.g.lpw;
  const int blocks = (warps * 32 + kLineThreads - 1) / kLineThreads;
  switch (a.g.n) {
    case 1: k_apply_M<R, 1><<<blocks, kLineThreads, 0, s>>>(a); break;
    case 2: k_apply_M<R, 2><<<blocks, kLineThreads, 0, s>>>(a); break;
    case 3: k_apply_M<R, 3><<<blocks, kLineThreads, 0, s>>>(a); break;
    case 4: k_apply_M<R, 4><<<blocks, kLineThreads, 0, s>>>(a); break;
    default: throw Error(1, "unsupported sites per lane");
  }
  WF_CUDA(cudaGetLastError());
}
template void launch_apply_M<float>(const MArgs<float>&, cudaStream_t);
template void launch_apply_M<double>(const MArgs<double>&, cudaStream_t);

}  // namespace wf
