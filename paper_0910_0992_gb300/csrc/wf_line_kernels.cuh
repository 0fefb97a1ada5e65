// Line kernels as templates: the bodies behind k_line (C_L / C_R / T^-1 / T^-dag and the fused
// hop + time-line steps of the Schur operator; see wf_kernels.cu for the operations) and the
// Wilson matrix kernel k_apply_M, templated on the sites per lane they hold in registers (NM:
// NMAX for lines of up to 128 slots, NMAX_LONG for longer ones). Included by wf_kernels.cu (the
// launchers for NM = NMAX) and by wf_kernels_long_f32.cu / wf_kernels_long_f64.cu (the long-line
// launchers, compiled apart so that the builds run in parallel).
#pragma once

#include "wf_internal.h"
#include "wf_line.cuh"

namespace wf {

constexpr int kLineThreads = 128;
#ifndef WF_LINE_MINB
#define WF_LINE_MINB 3
#endif
// resident CTAs per SM the line kernels are compiled for (3: 168 registers; measured best
// on GB300 against 1 and 4, where 4 spills)
template <typename R, bool AX, bool FWD, int NM>
__device__ __forceinline__ void solve_half(Vec3<R> (&v)[NM][4], int s0, const LineArgs<R>& A, int l, int jj) {
  constexpr int NS = sizeof(R) == 4 ? 2 : 1;
  const Geom& g = A.g;
#pragma unroll
  for (int sp = 0; sp < 2; sp += NS) {
    Vec3<R> w[NM][NS];
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
      for (int s = 0; s < NS; ++s) w[m][s] = v[m][s0 + sp + s];
    if (AX)
      tline_solve_axial<R, NS, FWD>(w, A.pl + (size_t)l * 9, A.lamb + (size_t)l * 9, g, jj, A.inv_mu, A.bc);
    else
      tline_solve_general<R, NS, FWD>(w, A.ut + (size_t)l * NLINK_C * g.tp,
                                      (FWD ? A.lamf : A.lamb) + (size_t)l * 9, g, jj, A.inv_mu, A.bc);
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
      for (int s = 0; s < NS; ++s) v[m][s0 + sp + s] = w[m][s];
  }
}

template <typename R, bool AX, int NM>
__device__ __forceinline__ void apply_op(int op, Vec3<R> (&v)[NM][4], int s0, const LineArgs<R>& A, int l, int jj) {
  if (op == OP_FWD)
    solve_half<R, AX, true>(v, s0, A, l, jj);
  else if (op == OP_BWD)
    solve_half<R, AX, false>(v, s0, A, l, jj);
}

// SRC, OPU, OPL < 0: taken from the arguments at run time
#ifndef WF_LINE_MINB_F64
#define WF_LINE_MINB_F64 3
#endif
template <typename R>
struct LineMinBlocks {
  static constexpr int value = sizeof(R) == 4 ? WF_LINE_MINB : WF_LINE_MINB_F64;
};

// The kernel body for block blk of a launch over one lattice (see k_line and k_line_multi).
template <typename R, bool AX, int SRC, int OPU, int OPL, bool H = false, int NM = NMAX>
__device__ __forceinline__ void line_body(const LineArgs<R>& A, int blk) {
  static_assert(!H || SRC == SRC_LOAD, "FP16 storage: the line kernel loads its own site only");
  const Geom& g = A.g;
  const int src = SRC >= 0 ? SRC : A.src;
  const int opu = OPU >= 0 ? OPU : A.opu;
  const int opl = OPL >= 0 ? OPL : A.opl;
  const int lane = threadIdx.x & 31;
  const int warp = (blk * (int)blockDim.x + (int)threadIdx.x) >> 5;
  const int lg_raw = warp * g.lpw + lane / g.lpl;
  const bool active = lg_raw < A.nrhs * g.Nl;
  const int lg = active ? lg_raw : 0;  // idle lanes still join the warp shuffles
  int rhs, l;
  line_rhs(lg, A.nrhs, g, rhs, l);
  const int jj = lane % g.lpl;
  const int tp = g.tp, n = g.n;
  const size_t base = ((size_t)rhs * g.Nl + l) * NSPIN_C * tp;
  if (A.active && g.lpw == 1 && !A.active[rhs]) return;  // one line per warp: the whole warp leaves

  Vec3<R> v[NM][4];
  if (src == SRC_HOP) {
    hop_spatial<R>(v, A, rhs, l, jj);
  } else {
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const int sl = m * g.lpl + jj;
      const bool ok = m < n;
      const bool up = ok && opu != OP_SKIP, lo = ok && opl != OP_SKIP;
      v[m][0] = up ? ldv<R, H>(A.src_up, base, tp, sl) : vzero<R>();
      v[m][1] = up ? ldv<R, H>(A.src_up, base + 3 * tp, tp, sl) : vzero<R>();
      v[m][2] = lo ? ldv<R, H>(A.src_lo, base, tp, sl) : vzero<R>();
      v[m][3] = lo ? ldv<R, H>(A.src_lo, base + 3 * tp, tp, sl) : vzero<R>();
    }
  }
  if (A.xpre) {
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      if (m >= n) continue;
#pragma unroll
      for (int s = 0; s < 4; ++s)
        v[m][s] = vaxpy(A.apre, v[m][s], ldv<R, H>(A.xpre, base + 3 * s * tp, tp, m * g.lpl + jj));
    }
  }

  apply_op<R, AX>(opu, v, 0, A, l, jj);
  apply_op<R, AX>(opl, v, 2, A, l, jj);

  R nrm = R(0);
  const bool want_norm = A.norm2 != nullptr;
  if (active) {
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      if (m >= n) continue;
      const int sl = m * g.lpl + jj;
      const bool valid = jj * n + m < g.T;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int op = h ? opl : opu;
        if (op == OP_SKIP) continue;
        const int dh = A.swap_out ? 1 - h : h;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int comp0 = dh * 6 + s * 3;
          Vec3<R> val = valid ? v[m][2 * h + s] : vzero<R>();
          if (A.xpost) val = vaxpy(A.apost, val, ldv<R, H>(A.xpost, base + comp0 * tp, tp, sl));
          stv<R, H>(A.out, base + comp0 * tp, tp, sl, val);
          if (want_norm) nrm += vnorm2(val);
        }
      }
    }
  }
  if (want_norm) {
    // lanes of one line share rhs; reduce over the warp per line group, one atomic per line
    double dn = (double)nrm;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_down_sync(0xffffffffu, dn, o);
      if (o < g.lpl) dn += other;
    }
    if (active && jj == 0) atomicAdd(A.norm2 + rhs, dn);
  }
}

template <typename R, bool AX, int SRC, int OPU, int OPL, bool H = false, int NM = NMAX>
__global__ void __launch_bounds__(kLineThreads, LineMinBlocks<R>::value) k_line(const LineArgs<R> A) {
  line_body<R, AX, SRC, OPU, OPL, H, NM>(A, blockIdx.x);
}

// one launch over a ragged batch of lattices (MultiLineArgs, wf_line.cuh)
template <typename R, bool AX, int SRC, int OPU, int OPL>
__global__ void __launch_bounds__(kLineThreads, LineMinBlocks<R>::value) k_line_multi(const MultiLineArgs<R> M) {
  int k = 0;
  while (k + 1 < M.n && (int)blockIdx.x >= M.blk0[k + 1]) ++k;
  line_body<R, AX, SRC, OPU, OPL>(M.a[k], (int)blockIdx.x - M.blk0[k]);
}

template <typename R>
inline int line_blocks(const LineArgs<R>& a) {
  const int lines = a.nrhs * a.g.Nl;
  const int warps = (lines + a.g.lpw - 1) / a.g.lpw;
  return (warps * 32 + kLineThreads - 1) / kLineThreads;
}

// ----------------------------------------------------------------------------
// Wilson matrix M = mu - D_t - D_s / gamma_f (§II, Eq. for M) on the output parity:
// out_p = mu psi_p - D_t psi_p - D_s psi_q / gamma_f   (or x + a * that).
// Dirac-Pauli basis: P_- = (1 - gamma_t)/2 keeps spins 2-3, P_+ spins 0-1, so
// D_t psi(t) = P_- U_t(t) psi(t+1) + P_+ U_t^dag(t-1) psi(t-1), sign bc across the wrap.
// In the axial frame U_t(t) = 1 except U_t(N_t-1) = P.
// ----------------------------------------------------------------------------
template <typename R, bool AX, int NM>
__global__ void __launch_bounds__(kLineThreads) k_apply_M(const MArgs<R> A) {
  const Geom& g = A.g;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lg = warp * g.lpw + lane / g.lpl;
  if (lg >= A.nrhs * g.Nl) return;
  int rhs, l;
  line_rhs(lg, A.nrhs, g, rhs, l);
  const int jj = lane % g.lpl;
  const int tp = g.tp, T = g.T, n = g.n;
  const size_t base = ((size_t)rhs * g.Nl + l) * NSPIN_C * tp;

  LineArgs<R> H;
  H.g = g;
  H.parity = A.parity;
  H.src_up = A.psi_q + (A.swap ? 6 * tp : 0);
  H.src_lo = A.psi_q + (A.swap ? 0 : 6 * tp);
  H.us_out = A.us_out;
  H.us_nbr = A.us_nbr;
  Vec3<R> h[NM][4];
  hop_spatial<R>(h, H, rhs, l, jj);

  const Cx<R>* ut_line = AX ? nullptr : A.ut + (size_t)l * NLINK_C * tp;
  const Cx<R>* pp = A.psi_p + base;
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    if (m >= n) continue;
    const int t = jj * n + m;
    const int sl = m * g.lpl + jj;
    Vec3<R> res[4];
    if (t < T) {
      const int tf = t == T - 1 ? 0 : t + 1;
      const int tb = t == 0 ? T - 1 : t - 1;
      const R sf = t == T - 1 ? A.bc : R(1);
      const R sb = t == 0 ? A.bc : R(1);
      const int slf = slot_of(g, tf), slb = slot_of(g, tb);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int sr = A.swap ? (s + 2) % 4 : s;  // spin read for result spin s
        Vec3<R> nb = ldvec(pp + 3 * sr * tp, tp, s < 2 ? slb : slf);
        Vec3<R> dt;
        if (AX) {
          if (s < 2 && t == 0)
            dt = matvec_dag(ldmat(A.pl + (size_t)l * 9, 1, 0), nb);
          else if (s >= 2 && t == T - 1)
            dt = matvec(ldmat(A.pl + (size_t)l * 9, 1, 0), nb);
          else
            dt = nb;
        } else {
          dt = s < 2 ? matvec_dag(ldmat(ut_line, tp, slb), nb) : matvec(ldmat(ut_line, tp, sl), nb);
        }
        const R sg = s < 2 ? sb : sf;
        Vec3<R> r = vscale(A.mu, ldvec(pp + 3 * sr * tp, tp, sl));
        r = vaxpy(-sg, dt, r);
        res[s] = vaxpy(-A.inv_gf, h[m][s], r);
      }
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s) res[s] = vzero<R>();
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int so = A.swap ? (s + 2) % 4 : s;
      Vec3<R> val = res[s];
      if (A.x) val = vaxpy(A.a, val, ldvec(A.x + base + 3 * so * tp, tp, sl));
      stvec(A.out + base + 3 * so * tp, tp, sl, val);
    }
  }
}

}  // namespace wf
