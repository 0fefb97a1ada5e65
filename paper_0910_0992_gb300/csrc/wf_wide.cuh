// Wide line kernels for the axial frame: one thread per time site.
//
// The line kernel of wf_kernels.cu gives each lane n sites of a line (n = 4 for N_t = 128).
// Its per-thread state -- n spinors of accumulator plus one direction's hop operands for n
// sites -- needs about 170 registers, which leaves 12 warps per SM, too few loads in flight to
// cover HBM latency (measured near 45 % of DRAM bandwidth, stalled on long scoreboard). Here
// thread q of a line owns the single slot q of the line layout, i.e. the site
//     t = n j + m   for slot q = m lpl + j,
// so that every warp-wide load is one contiguous run of 32 elements, as in k_line. (A map
// t = q, warps on consecutive times, touches four 64-byte runs per load and saturated the L1
// data pipe instead.) The hop keeps one spinor of accumulator live, so several times more
// warps fit per SM.
//
// The time-line solves of the axial frame (§II.C, App. C: U_t = 1 on the line except the
// boundary link P) are the recurrences
//     T^-dag: e(t) = mu^-1 (v(t) + e(t - 1)),   T^-1: e(t) = mu^-1 (v(t) + e(t + 1)),
// closed at the wrap: the value entering the line is s K^dag C (T^-dag) or s K C (T^-1), with
// K = P Lambda the per-line wrap matrix and C the line's composite with nothing entering.
// Every site is the affine map e -> c + a e (c = mu^-1 v, a = mu^-1; the identity on padding).
// The n sites of group j (t = n j .. n j + n - 1) sit in n different warps at lane j; their
// maps are composed through shared memory, then the lpl group composites by a Kogge-Stone
// shuffle scan over the lanes. A site's result is its in-group composite applied to the value
// entering its group. One barrier serves both spin halves. Memory layout, arguments and
// results are those of k_line.
#pragma once

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "wf_internal.h"
#include "wf_line.cuh"

namespace wf {

namespace wide {

constexpr int kWideCta = 128;  // threads per CTA
constexpr int kMapFields = 13;  // c (two spins x three colours, complex) and a
// resident CTAs per SM the kernels are compiled for. FP32: 7 (72 registers, no spills), measured
// on GB300 with 12 sources 1.07-1.15x faster than 5 (96 registers) and level with 8 (spills)
#ifndef WF_WIDE_MINB_F32
#define WF_WIDE_MINB_F32 7
#endif
#ifndef WF_WIDE_MINB_F64
#define WF_WIDE_MINB_F64 3
#endif
#ifndef WF_EARLY_X
#define WF_EARLY_X 1
#endif
#ifndef WF_WIDE_MINB_F32_C
#define WF_WIDE_MINB_F32_C WF_WIDE_MINB_F32
#endif
// KC: the K-c variant (its own bound: it holds the early-loaded post-axpy operand)
template <typename R, bool KC>
struct WideMinBlocks {
  static constexpr int value = WF_WIDE_MINB_F64;
};
template <bool KC>
struct WideMinBlocks<float, KC> {
  static constexpr int value = KC ? WF_WIDE_MINB_F32_C : WF_WIDE_MINB_F32;
};
#ifndef WF_WIDE_MINB_DF
#define WF_WIDE_MINB_DF 3
#endif
template <bool KC>
struct WideMinBlocks<df64, KC> {
  static constexpr int value = WF_WIDE_MINB_DF;
};

constexpr unsigned kFull = 0xffffffffu;

// the six neighbour lines of line l: from the table if the caller passed one
template <typename R>
__device__ __forceinline__ void neighbours(const LineArgs<R>& A, int l, int (&nb)[6]) {
  if (A.nbr) {
    const int2* t = reinterpret_cast<const int2*>(A.nbr + (size_t)l * 6);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int2 v = t[i];
      nb[2 * i] = v.x;
      nb[2 * i + 1] = v.y;
    }
  } else {
    neighbour_lines(A.g, A.parity, l, nb);
  }
}


// the affine map e -> c + a e on a spin half (two spins)
template <typename R>
struct HalfMap {
  Vec3<R> c[2];
  R a;
};

template <typename R>
__device__ __forceinline__ HalfMap<R> identity_map() {
  HalfMap<R> m;
  m.c[0] = vzero<R>();
  m.c[1] = vzero<R>();
  m.a = R(1);
  return m;
}

// later o earlier: apply `earlier` first, then `later`
template <typename R>
__device__ __forceinline__ HalfMap<R> compose(const HalfMap<R>& later, const HalfMap<R>& earlier) {
  HalfMap<R> r;
  r.c[0] = vaxpy(later.a, earlier.c[0], later.c[0]);
  r.c[1] = vaxpy(later.a, earlier.c[1], later.c[1]);
  r.a = later.a * earlier.a;
  return r;
}

template <typename R>
__device__ __forceinline__ HalfMap<R> shfl_map(const HalfMap<R>& m, int d, int width, bool up) {
  HalfMap<R> r;
  r.c[0] = up ? vshfl_up(m.c[0], d, width) : vshfl_down(m.c[0], d, width);
  r.c[1] = up ? vshfl_up(m.c[1], d, width) : vshfl_down(m.c[1], d, width);
  r.a = up ? shfl_up_r(m.a, d, width) : shfl_down_r(m.a, d, width);
  return r;
}

// shared-memory image of one map per thread, field-major (conflict-free)
template <typename R>
struct MapStore {
  R f[kMapFields][kWideCta];
};

template <typename R>
__device__ __forceinline__ void put_map(MapStore<R>& S, int q, const HalfMap<R>& m) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      S.f[6 * s + 2 * k][q] = m.c[s].c[k].re;
      S.f[6 * s + 2 * k + 1][q] = m.c[s].c[k].im;
    }
  S.f[12][q] = m.a;
}

template <typename R>
__device__ __forceinline__ HalfMap<R> get_map(const MapStore<R>& S, int q) {
  HalfMap<R> m;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int k = 0; k < 3; ++k) m.c[s].c[k] = mk<R>(S.f[6 * s + 2 * k][q], S.f[6 * s + 2 * k + 1][q]);
  m.a = S.f[12][q];
  return m;
}

// The same hop with the direction loop kept rolled (one copy of the SU(3) code): the backward
// hop uses the conjugate-transposed link, the projection and reconstruction signs are selected
// per direction, and the common factor 1/2 of the projectors is applied once at the end (exact).
// Used for double-float, whose unrolled hop overflows the instruction cache.
template <typename R, int TPC>
__device__ __forceinline__ void hop_site_rolled(Vec3<R> (&h)[4], const LineArgs<R>& A, int rhs, int l, int sl) {
  const Geom& g = A.g;
  const int tp = TPC ? TPC : g.tp, Nl = g.Nl;
  int nb[6];
  neighbours(A, l, nb);
#pragma unroll
  for (int s = 0; s < 4; ++s) h[s] = vzero<R>();
  constexpr int LNC = SpatialLinkNC<R>::value;
#pragma unroll 1
  for (int d = 0; d < 6; ++d) {
    const int k = d >> 1, dir = d & 1;  // dir 0: forward (x + k), 1: backward (x - k)
    const int ln = nb[d];
    const size_t sb = (size_t)(rhs * Nl + ln) * NSPIN_C * tp;
    const Cx<R>* lk = dir == 0 ? A.us_out + (size_t)(k * Nl + l) * LNC * tp
                               : A.us_nbr + (size_t)(k * Nl + ln) * LNC * tp;
    Mat3<R> U = ldlink(lk, tp, sl);
    if (dir) U = dagger(U);
    const Vec3<R> u0 = ldvec(A.src_up + sb, tp, sl), u1 = ldvec(A.src_up + sb + 3 * tp, tp, sl);
    const Vec3<R> d0 = ldvec(A.src_lo + sb, tp, sl), d1 = ldvec(A.src_lo + sb + 3 * tp, tp, sl);
    Vec3<R> s0, s1;
    isigma(k, d0, d1, s0, s1);
    if (dir) {
      s0 = vneg(s0);
      s1 = vneg(s1);
    }
    const Vec3<R> w0 = matvec(U, vadd(u0, s0)), w1 = matvec(U, vadd(u1, s1));
    h[0] = vadd(h[0], w0);
    h[1] = vadd(h[1], w1);
    Vec3<R> r0, r1;
    isigma(k, w0, w1, r0, r1);
    if (!dir) {
      r0 = vneg(r0);
      r1 = vneg(r1);
    }
    h[2] = vadd(h[2], r0);
    h[3] = vadd(h[3], r1);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) h[s] = vscale(R(0.5), h[s]);
}

template <typename R>
__device__ __forceinline__ HalfMap<R> site_map(const Vec3<R>& v0, const Vec3<R>& v1, bool valid, R inv_mu) {
  HalfMap<R> m;
  m.c[0] = valid ? vscale(inv_mu, v0) : vzero<R>();
  m.c[1] = valid ? vscale(inv_mu, v1) : vzero<R>();
  m.a = valid ? inv_mu : R(1);
  return m;
}

// Solve one half after all site maps of the CTA are in S (thread q0 + mm lpl holds site
// mm of this thread's group). FWD: T^-dag, time increasing; else T^-1, time decreasing.
template <typename R, bool FWD>
__device__ __forceinline__ void solve_half_wide(Vec3<R>& v0, Vec3<R>& v1, const MapStore<R>& S, bool member, int q0,
                                                int m, int n, int lpl, int j, bool valid,
                                                const Cx<R>* __restrict__ K_line, R bc) {
  // composites within the group: up to this thread's site, and over the whole group
  HalfMap<R> incl = identity_map<R>(), grp = identity_map<R>();
  if (member) {
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
      if (i >= n) break;
      const int mm = FWD ? i : n - 1 - i;
      grp = compose(get_map(S, q0 + mm * lpl), grp);
      if (mm == m) incl = grp;
    }
  }
  // scan of the group composites over the lanes of the line, in time order
  HalfMap<R> gs = grp;
  for (int d = 1; d < lpl; d <<= 1) {
    const HalfMap<R> o = shfl_map(gs, d, lpl, FWD);
    if (FWD ? j >= d : j + d < lpl) gs = compose(gs, o);
  }
  // the line's composite sits at its last group in time order; the wrap value enters the first
  Vec3<R> e[2];
  {
    const int last = FWD ? lpl - 1 : 0;
    const Vec3<R> C0 = vshfl_idx(gs.c[0], last, lpl), C1 = vshfl_idx(gs.c[1], last, lpl);
    const Mat3<R> K = ldmat(K_line, 1, 0);
    e[0] = vscale(bc, FWD ? matvec_dag(K, C0) : matvec(K, C0));
    e[1] = vscale(bc, FWD ? matvec_dag(K, C1) : matvec(K, C1));
  }
  // value entering this group: the composite of the groups before it, applied to the wrap
  const HalfMap<R> prev = shfl_map(gs, 1, lpl, FWD);
  if (FWD ? j > 0 : j < lpl - 1) {
    e[0] = vaxpy(prev.a, e[0], prev.c[0]);
    e[1] = vaxpy(prev.a, e[1], prev.c[1]);
  }
  v0 = valid ? vaxpy(incl.a, e[0], incl.c[0]) : vzero<R>();
  v1 = valid ? vaxpy(incl.a, e[1], incl.c[1]) : vzero<R>();
}

// D_s (the spatial hop of hop_spatial, wf_line.cuh) at one site of line l
template <typename R, int TPC, bool H = false>
__device__ __forceinline__ void hop_site(Vec3<R> (&h)[4], const LineArgs<R>& A, int rhs, int l, int sl) {
  const Geom& g = A.g;
  const int tp = TPC ? TPC : g.tp, Nl = g.Nl;
  int nb[6];
  neighbours(A, l, nb);
#pragma unroll
  for (int s = 0; s < 4; ++s) h[s] = vzero<R>();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {  // 0: forward (x + k), 1: backward (x - k)
      const int ln = nb[2 * k + dir];
      const size_t sb = (size_t)(rhs * Nl + ln) * NSPIN_C * tp;
      constexpr int LNC = SpatialLinkNC<R>::value;
      const Cx<R>* lk = dir == 0 ? A.us_out + (size_t)(k * Nl + l) * LNC * tp
                                 : A.us_nbr + (size_t)(k * Nl + ln) * LNC * tp;
      const Vec3<R> u0 = ldv<R, H>(A.src_up, sb, tp, sl), u1 = ldv<R, H>(A.src_up, sb + 3 * tp, tp, sl);
      const Vec3<R> d0 = ldv<R, H>(A.src_lo, sb, tp, sl), d1 = ldv<R, H>(A.src_lo, sb + 3 * tp, tp, sl);
      const Mat3<R> U = ldlink(lk, tp, sl);
      Vec3<R> s0, s1;
      isigma(k, d0, d1, s0, s1);
      Vec3<R> h0, h1;  // the projectors' factor 1/2 is applied once at the end (exact)
      if (dir == 0) {
        h0 = vadd(u0, s0);
        h1 = vadd(u1, s1);
      } else {
        h0 = vaxpy(R(-1), s0, u0);
        h1 = vaxpy(R(-1), s1, u1);
      }
      const Vec3<R> w0 = dir == 0 ? matvec(U, h0) : matvec_dag(U, h0);
      const Vec3<R> w1 = dir == 0 ? matvec(U, h1) : matvec_dag(U, h1);
      h[0] = vadd(h[0], w0);
      h[1] = vadd(h[1], w1);
      Vec3<R> r0, r1;
      isigma(k, w0, w1, r0, r1);
      if (dir == 0) {
        h[2] = vaxpy(R(-1), r0, h[2]);
        h[3] = vaxpy(R(-1), r1, h[3]);
      } else {
        h[2] = vadd(h[2], r0);
        h[3] = vadd(h[3], r1);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) h[s] = vscale(R(0.5), h[s]);
}

// Time-line solve of one spin of a lane group's four sites (tp = 128: n = 4, 32 lanes), three
// colours held by the thread: the recurrence over the four sites in registers, the group
// composites scanned over the 32 lanes, the wrap through K within the warp.
template <typename R, bool FWD>
__device__ __forceinline__ void spin_solve4(Vec3<R> (&w)[4], int j, int T, const Cx<R>* __restrict__ K_line,
                                            R inv_mu, R bc) {
  Vec3<R> c = vzero<R>();
  R a = R(1);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int mm = FWD ? i : 3 - i;
    if (4 * j + mm >= T) continue;  // padding: identity
    c = vscale(inv_mu, vadd(w[mm], c));
    a *= inv_mu;
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const R an = FWD ? shfl_up_r(a, d, 32) : shfl_down_r(a, d, 32);
    const Vec3<R> cn = FWD ? vshfl_up(c, d, 32) : vshfl_down(c, d, 32);
    if (FWD ? j >= d : j + d < 32) {
      c = vaxpy(a, cn, c);
      a *= an;
    }
  }
  // the line's composite is at its last lane in time order; the wrap value enters the first
  const Vec3<R> C = vshfl_idx(c, FWD ? 31 : 0, 32);
  const Mat3<R> K = ldmat(K_line, 1, 0);
  Vec3<R> e = vscale(bc, FWD ? matvec_dag(K, C) : matvec(K, C));
  const R ap = FWD ? shfl_up_r(a, 1, 32) : shfl_down_r(a, 1, 32);
  const Vec3<R> cp = FWD ? vshfl_up(c, 1, 32) : vshfl_down(c, 1, 32);
  if (FWD ? j > 0 : j < 31) e = vaxpy(ap, e, cp);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int mm = FWD ? i : 3 - i;
    if (4 * j + mm >= T) {
      w[mm] = vzero<R>();
      continue;
    }
    e = vscale(inv_mu, vadd(w[mm], e));
    w[mm] = e;
  }
}

// one atomic per line for |out|^2 (lines of whole warps)
template <typename R>
__device__ __forceinline__ void line_norm_whole_warps(double* nrm_s, R nrm, int q, int tp, int li, int sl, bool line_ok,
                                                      double* norm2, int rhs) {
  double dn = (double)nrm;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dn += __shfl_down_sync(kFull, dn, o);
  if ((q & 31) == 0) nrm_s[q >> 5] = dn;
  __syncthreads();
  if (line_ok && sl == 0) {
    double sum = 0.0;
    for (int i = 0; i < tp / 32; ++i) sum += nrm_s[(li * tp >> 5) + i];
    atomicAdd(norm2 + rhs, sum);
  }
}

// SRC, OPU, OPL < 0: taken from the arguments at run time. TPC: the line length tp as a
// compile-time constant (128: n = 4 sites per group, 32 lanes, so that every load's component
// offset is an immediate), or 0 to read the layout at run time.
// The kernel body (wf_wide_body.inc) as a device function for block blk of one lattice's part of a
// multi-lattice launch; k_line_wide includes the same body directly.
template <typename R, int SRC, int OPU, int OPL, int TPC, bool H = false>
__device__ __forceinline__ void line_wide_body(const LineArgs<R>& A, int blk) {
#define WF_WIDE_BLOCK blk
#include "wf_wide_body.inc"
#undef WF_WIDE_BLOCK
}

template <typename R, int SRC, int OPU, int OPL, int TPC, bool H = false>
__global__ void __launch_bounds__(kWideCta, WideMinBlocks<R, SRC == SRC_HOP && OPU == OP_COPY>::value)
    k_line_wide(const LineArgs<R> A) {
#define WF_WIDE_BLOCK ((int)blockIdx.x)
#include "wf_wide_body.inc"
#undef WF_WIDE_BLOCK
}

// One launch over several lattices (a ragged batch): block b belongs to the lattice k with
// M.blk0[k] <= b < M.blk0[k + 1] and runs that lattice's arguments. TPC as for k_line_wide: the
// lattices of one launch share it (128-slot lines and the others launch apart).
template <typename R, int SRC, int OPU, int OPL, int TPC>
__global__ void __launch_bounds__(kWideCta, WideMinBlocks<R, SRC == SRC_HOP && OPU == OP_COPY>::value)
    k_line_wide_multi(const __grid_constant__ MultiLineArgs<R> M) {
  int k = 0;
  while (k + 1 < M.n && (int)blockIdx.x >= M.blk0[k + 1]) ++k;
  line_wide_body<R, SRC, OPU, OPL, TPC>(M.a[k], (int)blockIdx.x - M.blk0[k]);
}

}  // namespace wide

// K-b or K-c (LK_SCHUR_B / LK_SCHUR_C) over a ragged batch of lattices, each with its own
// arguments (traversal and neighbour tables attached): the lattices with 128-slot lines in
// launches of up to kMaxLattices, the others likewise
template <typename R>
void launch_line_wide_multi(const std::vector<LineArgs<R>>& as, int kind, cudaStream_t s) {
  if (kind != LK_SCHUR_B && kind != LK_SCHUR_C) throw Error(1, "multi-lattice wide kernel: K-b or K-c only");
  for (int compiled = 1; compiled >= 0; --compiled) {
    std::vector<const LineArgs<R>*> sel;
    for (const LineArgs<R>& a : as) {
      if (!wide_supported(a.g) || a.h16 || !a.order || !a.nbr)
        throw Error(1, "multi-lattice wide kernel: supported layouts, FP32 storage, traversal tables");
      const bool is128 = a.g.tp == 128 && a.g.n == 4 && a.g.lpl == 32;
      if (is128 == (compiled == 1)) sel.push_back(&a);
    }
    for (size_t first = 0; first < sel.size(); first += kMaxLattices) {
      MultiLineArgs<R> M;
      std::memset(&M, 0, sizeof(M));
      M.n = (int)std::min<size_t>(kMaxLattices, sel.size() - first);
      int blocks = 0;
      for (int k = 0; k < M.n; ++k) {
        const LineArgs<R>& a = *sel[first + k];
        M.a[k] = a;
        M.blk0[k] = blocks;
        const int LPC = wide::kWideCta / a.g.tp;
        blocks += (a.nrhs * a.g.Nl + LPC - 1) / LPC;
      }
      M.blk0[M.n] = blocks;
      if (blocks == 0) continue;
#define WF_KWM(OPUV, TPCV) wide::k_line_wide_multi<R, SRC_HOP, OPUV, OP_BWD, TPCV><<<blocks, wide::kWideCta, 0, s>>>(M)
      if (kind == LK_SCHUR_B) {
        if (compiled)
          WF_KWM(OP_FWD, 128);
        else
          WF_KWM(OP_FWD, 0);
      } else {
        if (compiled)
          WF_KWM(OP_COPY, 128);
        else
          WF_KWM(OP_COPY, 0);
      }
#undef WF_KWM
      WF_CUDA(cudaGetLastError());
    }
  }
}

// launch of the kernel variant for `kind` (LineKind) over all lines of all right-hand sides;
// instantiated for float in wf_wide.cu and for double-float in wf_wide_df.cu
template <typename R>
void launch_line_wide(const LineArgs<R>& a, int kind, cudaStream_t s) {
  if (!wide_supported(a.g)) throw Error(1, "wide line kernel: unsupported line layout");
  const int LPC = wide::kWideCta / a.g.tp;
  const int lines = a.nrhs * a.g.Nl;
  const int blocks = (lines + LPC - 1) / LPC;
  const bool t128 = a.g.tp == 128 && a.g.n == 4 && a.g.lpl == 32;
  constexpr bool kF32 = std::is_same<R, float>::value;
  if (a.h16 && !kF32) throw Error(1, "wide line kernel: FP16 storage needs FP32 arithmetic");
#define WF_KW(SRCV, OPUV, OPLV)                                                                   \
  do {                                                                                            \
    constexpr bool kH = kF32 && (SRCV) == SRC_HOP; /* FP16 storage: the hop kernels K-b, K-c */  \
    if (a.h16) {                                                                                  \
      if (!kH) throw Error(1, "wide line kernel: FP16 storage only for the hop kernels");         \
      if (t128)                                                                                   \
        wide::k_line_wide<R, SRCV, OPUV, OPLV, 128, kH><<<blocks, wide::kWideCta, 0, s>>>(a);     \
      else                                                                                        \
        wide::k_line_wide<R, SRCV, OPUV, OPLV, 0, kH><<<blocks, wide::kWideCta, 0, s>>>(a);       \
    } else if (t128) {                                                                            \
      wide::k_line_wide<R, SRCV, OPUV, OPLV, 128><<<blocks, wide::kWideCta, 0, s>>>(a);           \
    } else {                                                                                      \
      wide::k_line_wide<R, SRCV, OPUV, OPLV, 0><<<blocks, wide::kWideCta, 0, s>>>(a);             \
    }                                                                                             \
  } while (0)
  switch (kind) {
    case LK_SCHUR_A: WF_KW(SRC_LOAD, OP_FWD, OP_SKIP); break;
    case LK_SCHUR_B: WF_KW(SRC_HOP, OP_FWD, OP_BWD); break;
    case LK_SCHUR_C: WF_KW(SRC_HOP, OP_COPY, OP_BWD); break;
    default: WF_KW(-1, -1, -1); break;
  }
#undef WF_KW
  WF_CUDA(cudaGetLastError());
}

}  // namespace wf
