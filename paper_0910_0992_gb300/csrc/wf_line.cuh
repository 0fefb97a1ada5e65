// Time-line solves (T^-1, T^-dag) and the spatial hop D_s on the line layout.
//
// T^-1 (§II.A): psi(t) = (eta(t) + U_0(t) psi(t+1)) / mu for t = N_t-1 .. 0, with the
// wrap psi(N_t) = s psi(0). T^-dag: psi(t) = (eta(t) + U_0^dag(t-1) psi(t-1)) / mu for
// t = 0 .. N_t-1, with psi(-1) = s psi(N_t-1).
//
// The paper closes the wrap-around with the Sherman-Morrison-Woodbury correction
// chi = T_0^-1 eta, q = Lambda W^dag chi, psi = chi - X q. Here the same exact result is
// reached warp-parallel: each lane owns n consecutive times and turns them into one affine
// map psi_out = c + G psi_in (c: open-boundary solution of its segment; G: product of
// U_0 / mu over the segment); a Kogge-Stone scan of these maps over the lanes of the line
// gives every lane the map from the line's open end to its segment; the wrap is closed with
// the per-line Lambda = (I - s mu^-N_t P)^-1 (P the Polyakov product, precomputed in FP64
// at gauge load, §II.A step 1(b)); each lane then re-runs its n steps from its true
// boundary value. Every input is read once and every output written once.
//
// Two frames:
// * general: U_0 as given; G is a 3x3 matrix (tline_solve_general).
// * axial: the gauge field was rotated once at load so that U_0(t) = 1 for t < N_t - 1
//   and U_0(N_t - 1) = P (§II.C, "axial gauge"; App. C). Then every lane's G is the scalar
//   mu^-k, the scan composes scalars and vectors only, no U_0 is read, and P enters once,
//   at the wrap (tline_solve_axial).
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "wf_common.cuh"

namespace wf {

constexpr int NMAX = 4;       // sites per lane of the fast kernels (T <= 32 * NMAX)
constexpr int NMAX_LONG = 8;  // sites per lane of the n-sites-per-lane kernels' long-line variant (T <= 256)

enum LineOp { OP_COPY = 0, OP_FWD = 1, OP_BWD = 2, OP_SKIP = 3 };
enum LineSrc { SRC_LOAD = 0, SRC_HOP = 1 };

template <typename R>
struct LineArgs {
  Geom g;
  int parity;   // 3-D parity of the output lines
  int nrhs;
  int opu, opl; // LineOp for the upper (P_+) and lower (P_-) spin halves (runtime-op kernel)
  int src;      // LineSrc (runtime-op kernel)
  // Spinor sources. SRC_LOAD reads the output site itself; SRC_HOP reads the six
  // spatial neighbours (other parity). src_up / src_lo point at component 0 of the
  // half that supplies spins 0-1 / spins 2-3 (line stride 12 * tp).
  const Cx<R>* src_up;
  const Cx<R>* src_lo;
  // links: U_t of the output parity [Nl][9][tp] (general frame), the per-line boundary
  // link P [Nl][9] (axial frame), forward spatial links of the output parity and of the
  // neighbour parity, each [3][Nl][SpatialLinkNC][tp]
  const Cx<R>* ut;
  const Cx<R>* pl;
  const Cx<R>* us_out;
  const Cx<R>* us_nbr;
  const Cx<R>* lamb;  // Lambda for T^-1, [Nl][9]
  const Cx<R>* lamf;  // general frame: Lambda for T^-dag, [Nl][9]; axial frame: the wrap matrix
                      // K = P Lambda, [Nl][9] (T^-1 closes with K, T^-dag with K^dag)
  // pre-solve axpy: v <- xpre + apre * v (skipped if xpre == nullptr)
  const Cx<R>* xpre;
  R apre;
  // post-solve: out <- xpost + apost * result (plain store if xpost == nullptr)
  const Cx<R>* xpost;
  R apost;
  int swap_out;  // store the upper result into the lower half and vice versa
  int stream_out;  // store with the evict-first cache policy (the result is not read again soon)
  Cx<R>* out;    // [nrhs][Nl][12][tp]
  double* norm2; // if set: atomically add |stored result|^2 per rhs (FP64)
  R inv_mu, bc;
  int drop_job;  // TMA-fed kernel only: skip the bulk copy of this job (fault injection), -1: none
  int df;        // R = double only: compute in double-float (FP64 storage, FP32 arithmetic)
  // optional index tables (wide kernels; null: computed in the kernel): the (rhs, line) of every
  // traversal position [nrhs * Nl] (line_rhs), and the six neighbour lines of every output line
  // [Nl][6] (neighbour_lines, output parity)
  const int2* order;
  const int* nbr;
  int variant;  // FP32 axial hop kernels: 0 the built-in choice, 1 one thread per site, 2 n sites per lane,
                // 3 bulk-fed (wf_pipe.cu) with pipe_g sources per unit and pipe_ns stages
  int pipe_g, pipe_ns;
  // FP32 kernels only: the spinor fields (src_up, src_lo, xpre, xpost, out) hold FP16 (Cx16) data
  int h16;
  // if set: [nrhs] flags; right-hand sides whose flag is 0 are skipped (kernels whose CTA or
  // warp holds lines of one right-hand side only; their outputs for those sources are left as is)
  const int* active;
};

// Arguments of one launch over a ragged batch of lattices (kMaxLattices at most per launch): the
// per-lattice arguments and the first block of each lattice (blk0[n] = total blocks).
constexpr int kMaxLattices = 8;
template <typename R>
struct MultiLineArgs {
  int n;
  int blk0[kMaxLattices + 1];
  LineArgs<R> a[kMaxLattices];
};

// Order in which the line kernels visit (rhs, line) pairs. Right-hand sides are processed in
// groups of kRhsGroup; within a group every line is visited for all of the group's
// right-hand sides side by side, so the line's links are shared through L2 (measured: groups
// of all 12 sources beat groups of 4, whose links are re-read per group). Lines are visited in
// tiles of all x times g.by rows of y, each tile streamed along z: a neighbour line's spinor
// is then read again by the other hops of the stencil while still in L2 (reuse distance about
// Lh * by lines instead of Lh * L lines in lexicographic order; measured with 12 sources on
// 24^3 x 128: lexicographic order read the neighbour spinors about three times from DRAM).
#ifndef WF_RHS_GROUP
#define WF_RHS_GROUP 16
#endif
constexpr int kRhsGroup = WF_RHS_GROUP;

// traversal index -> (rhs, line); host and device (the wide kernels read it from a table)
__host__ __device__ __forceinline__ void line_rhs(int lg, int nrhs, const Geom& g, int& rhs, int& l) {
  const int per_group = kRhsGroup * g.Nl;
  const int grp = lg / per_group;
  const int r = lg - grp * per_group;
  const int left = nrhs - grp * kRhsGroup;
  const int gsize = left < kRhsGroup ? left : kRhsGroup;
  const int pos = r / gsize;  // position of the line in the tiled order
  rhs = grp * kRhsGroup + (r - pos * gsize);
  const int xh = pos % g.Lh;
  int u = pos / g.Lh;
  const int yy = u % g.by;
  u /= g.by;
  const int z = u % g.L;
  const int y = (u / g.L) * g.by + yy;
  l = xh + g.Lh * (y + g.L * z);
}

template <typename R>
__device__ __forceinline__ Mat3<R> ldmat(const Cx<R>* __restrict__ base, int tp, int slot) {
  Mat3<R> U;
#pragma unroll
  for (int k = 0; k < 9; ++k) U.e[k] = ldc(base + k * tp + slot);
  return U;
}

// a spatial link in its storage form (see SpatialLinkNC): 9 entries, or 2 rows and the
// third rebuilt as conj(row0 x row1)
template <typename R>
__device__ __forceinline__ Mat3<R> ldlink(const Cx<R>* __restrict__ base, int tp, int slot) {
  if constexpr (SpatialLinkNC<R>::value == 9) {
    return ldmat(base, tp, slot);
  }
  Mat3<R> U;
#pragma unroll
  for (int k = 0; k < 6; ++k) U.e[k] = ldc(base + k * tp + slot);
  const Cx<R>* a = U.e;
  const Cx<R>* b = U.e + 3;
  const Cx<R> c0 = cmul(a[1], b[2]) - cmul(a[2], b[1]);
  const Cx<R> c1 = cmul(a[2], b[0]) - cmul(a[0], b[2]);
  const Cx<R> c2 = cmul(a[0], b[1]) - cmul(a[1], b[0]);
  U.e[6] = mk<R>(c0.re, -c0.im);
  U.e[7] = mk<R>(c1.re, -c1.im);
  U.e[8] = mk<R>(c2.re, -c2.im);
  return U;
}

template <typename R>
__device__ __forceinline__ Vec3<R> ldvec(const Cx<R>* __restrict__ base, int tp, int slot) {
  Vec3<R> v;
#pragma unroll
  for (int k = 0; k < 3; ++k) v.c[k] = ldc(base + k * tp + slot);
  return v;
}

template <typename R>
__device__ __forceinline__ void stvec(Cx<R>* __restrict__ base, int tp, int slot, const Vec3<R>& v) {
#pragma unroll
  for (int k = 0; k < 3; ++k) stc(base + k * tp + slot, v.c[k]);
}

// single-use data: loads and stores with the evict-first ("streaming") cache policy, so that
// they do not push reusable neighbour lines and links out of L2
__device__ __forceinline__ Cx<float> ld_stream(const Cx<float>* p) {
  const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
  return mk<float>(v.x, v.y);
}
__device__ __forceinline__ Cx<double> ld_stream(const Cx<double>* p) {
  const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
  return mk<double>(v.x, v.y);
}
__device__ __forceinline__ Cx<df64> ld_stream(const Cx<df64>* p) {
  const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
  return mk<df64>(df_from_double(v.x), df_from_double(v.y));
}
__device__ __forceinline__ void st_stream(Cx<df64>* p, Cx<df64> z) {
  __stcs(reinterpret_cast<double2*>(p), make_double2(df_to_double(z.re), df_to_double(z.im)));
}
__device__ __forceinline__ void st_stream(Cx<float>* p, Cx<float> z) {
  __stcs(reinterpret_cast<float2*>(p), make_float2(z.re, z.im));
}
__device__ __forceinline__ void st_stream(Cx<double>* p, Cx<double> z) {
  __stcs(reinterpret_cast<double2*>(p), make_double2(z.re, z.im));
}
template <typename R>
__device__ __forceinline__ Vec3<R> ldvec_stream(const Cx<R>* __restrict__ base, int tp, int slot) {
  Vec3<R> v;
#pragma unroll
  for (int k = 0; k < 3; ++k) v.c[k] = ld_stream(base + k * tp + slot);
  return v;
}
template <typename R>
__device__ __forceinline__ void stvec_stream(Cx<R>* __restrict__ base, int tp, int slot, const Vec3<R>& v) {
#pragma unroll
  for (int k = 0; k < 3; ++k) st_stream(base + k * tp + slot, v.c[k]);
}

// ----------------------------------------------------------------------------
// Spinor storage: FP32 (Cx<float>, 8 B per complex) or FP16 (Cx16, one half2, 4 B per complex),
// both in the same element layout. FP32 kernels compute in FP32 either way; a kernel compiled
// for FP16 storage (H = true) converts at every spinor load and store. A field pointer keeps the
// type Cx<float>* in the argument structures; for FP16 fields it points at Cx16 data, so element
// offsets are added here, after the cast, never to the Cx<float>* itself.
// ----------------------------------------------------------------------------
struct __align__(4) Cx16 {
  __half2 v;
};

template <bool H>
__device__ __forceinline__ Cx<float> ld_sp(const Cx<float>* base, size_t off) {
  if constexpr (H) {
    const float2 f = __half22float2(reinterpret_cast<const Cx16*>(base)[off].v);
    return mk<float>(f.x, f.y);
  } else {
    return base[off];
  }
}
template <bool H>
__device__ __forceinline__ Cx<float> ld_sp_stream(const Cx<float>* base, size_t off) {
  if constexpr (H) {
    const unsigned u = __ldcs(reinterpret_cast<const unsigned*>(reinterpret_cast<const Cx16*>(base) + off));
    __half2 hv;
    memcpy(&hv, &u, sizeof(u));
    const float2 f = __half22float2(hv);
    return mk<float>(f.x, f.y);
  } else {
    return ld_stream(base + off);
  }
}
template <bool H>
__device__ __forceinline__ void st_sp(Cx<float>* base, size_t off, Cx<float> z) {
  if constexpr (H) {
    reinterpret_cast<Cx16*>(base)[off].v = __floats2half2_rn(z.re, z.im);
  } else {
    base[off] = z;
  }
}
template <bool H>
__device__ __forceinline__ void st_sp_stream(Cx<float>* base, size_t off, Cx<float> z) {
  if constexpr (H) {
    const __half2 hv = __floats2half2_rn(z.re, z.im);
    unsigned u;
    memcpy(&u, &hv, sizeof(u));
    __stcs(reinterpret_cast<unsigned*>(reinterpret_cast<Cx16*>(base) + off), u);
  } else {
    st_stream(base + off, z);
  }
}
// three colour components at element offsets off + k tp + slot
template <bool H>
__device__ __forceinline__ Vec3<float> ldvec_sp(const Cx<float>* base, size_t off, int tp, int slot) {
  Vec3<float> v;
#pragma unroll
  for (int k = 0; k < 3; ++k) v.c[k] = ld_sp<H>(base, off + (size_t)(k * tp + slot));
  return v;
}
template <bool H>
__device__ __forceinline__ Vec3<float> ldvec_sp_stream(const Cx<float>* base, size_t off, int tp, int slot) {
  Vec3<float> v;
#pragma unroll
  for (int k = 0; k < 3; ++k) v.c[k] = ld_sp_stream<H>(base, off + (size_t)(k * tp + slot));
  return v;
}
template <bool H>
__device__ __forceinline__ void stvec_sp(Cx<float>* base, size_t off, int tp, int slot, const Vec3<float>& v) {
#pragma unroll
  for (int k = 0; k < 3; ++k) st_sp<H>(base, off + (size_t)(k * tp + slot), v.c[k]);
}
template <bool H>
__device__ __forceinline__ void stvec_sp_stream(Cx<float>* base, size_t off, int tp, int slot, const Vec3<float>& v) {
#pragma unroll
  for (int k = 0; k < 3; ++k) st_sp_stream<H>(base, off + (size_t)(k * tp + slot), v.c[k]);
}

// spinor accessors of the line kernels: element offset off from a field's base pointer, in the
// precision R of the kernel or (H, R = float only) FP16 storage
template <typename R, bool H>
__device__ __forceinline__ Vec3<R> ldv(const Cx<R>* base, size_t off, int tp, int slot) {
  static_assert(!H || std::is_same<R, float>::value, "FP16 storage with FP32 arithmetic only");
  if constexpr (H) return ldvec_sp<true>(base, off, tp, slot);
  else return ldvec(base + off, tp, slot);
}
template <typename R, bool H>
__device__ __forceinline__ Vec3<R> ldv_stream(const Cx<R>* base, size_t off, int tp, int slot) {
  if constexpr (H) return ldvec_sp_stream<true>(base, off, tp, slot);
  else return ldvec_stream(base + off, tp, slot);
}
template <typename R, bool H>
__device__ __forceinline__ void stv(Cx<R>* base, size_t off, int tp, int slot, const Vec3<R>& v) {
  if constexpr (H) stvec_sp<true>(base, off, tp, slot, v);
  else stvec(base + off, tp, slot, v);
}
template <typename R, bool H>
__device__ __forceinline__ void stv_stream(Cx<R>* base, size_t off, int tp, int slot, const Vec3<R>& v) {
  if constexpr (H) stvec_sp_stream<true>(base, off, tp, slot, v);
  else stvec_stream(base + off, tp, slot, v);
}

template <typename R>
__device__ __forceinline__ Vec3<R> vzero() {
  Vec3<R> v;
#pragma unroll
  for (int k = 0; k < 3; ++k) v.c[k] = czero<R>();
  return v;
}

template <typename R>
__device__ __forceinline__ Vec3<R> vaxpy(R a, const Vec3<R>& x, const Vec3<R>& y) {  // y + a x
  Vec3<R> w;
#pragma unroll
  for (int k = 0; k < 3; ++k) w.c[k] = mk<R>(fma(a, x.c[k].re, y.c[k].re), fma(a, x.c[k].im, y.c[k].im));
  return w;
}

template <typename R>
__device__ __forceinline__ Vec3<R> vscale(R a, const Vec3<R>& x) {
  Vec3<R> w;
#pragma unroll
  for (int k = 0; k < 3; ++k) w.c[k] = a * x.c[k];
  return w;
}

template <typename R>
__device__ __forceinline__ Vec3<R> vneg(const Vec3<R>& x) {
  Vec3<R> w;
#pragma unroll
  for (int k = 0; k < 3; ++k) w.c[k] = mk<R>(-x.c[k].re, -x.c[k].im);
  return w;
}

template <typename R>
__device__ __forceinline__ Vec3<R> vadd(const Vec3<R>& x, const Vec3<R>& y) {
  Vec3<R> w;
#pragma unroll
  for (int k = 0; k < 3; ++k) w.c[k] = x.c[k] + y.c[k];
  return w;
}

// |x|^2 in the field's own precision (GB300's FP64 rate is far below its FP32 rate, so FP32
// kernels keep FP64 for the final cross-thread sums only)
template <typename R>
__device__ __forceinline__ R vnorm2(const Vec3<R>& x) {
  R s = R(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) s = fma(x.c[k].re, x.c[k].re, fma(x.c[k].im, x.c[k].im, s));
  return s;
}

template <typename R>
__device__ __forceinline__ Vec3<R> vshfl_down(const Vec3<R>& v, int d, int w) {
  Vec3<R> r;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.c[k] = shfl_down(v.c[k], d, w);
  return r;
}
template <typename R>
__device__ __forceinline__ Vec3<R> vshfl_up(const Vec3<R>& v, int d, int w) {
  Vec3<R> r;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.c[k] = shfl_up(v.c[k], d, w);
  return r;
}
template <typename R>
__device__ __forceinline__ Vec3<R> vshfl_idx(const Vec3<R>& v, int src, int w) {
  Vec3<R> r;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.c[k] = shfl_idx(v.c[k], src, w);
  return r;
}

// ----------------------------------------------------------------------------
// General frame: time-line solve of NS colour vectors per site on the lane's n sites.
// FWD = false: psi = T^-1 eta. FWD = true: psi = T^-dag eta. v holds eta on entry and
// psi on exit. ut_line: this line's U_t block ([9][tp]); lam: its Lambda. Warp-collective.
// ----------------------------------------------------------------------------
template <typename R, int NS, bool FWD, int NM>
__device__ __forceinline__ void tline_solve_general(Vec3<R> (&v)[NM][NS], const Cx<R>* __restrict__ ut_line,
                                                    const Cx<R>* __restrict__ lam, const Geom& g, int jj, R inv_mu,
                                                    R bc) {
  const int T = g.T, tp = g.tp, lpl = g.lpl, n = g.n;
  constexpr bool KEEPU = (sizeof(R) == 4);
  Mat3<R> Uk[KEEPU ? NM : 1];

  auto link_slot = [&](int m) {
    int t = jj * n + m;
    int tl = FWD ? (t == 0 ? T - 1 : t - 1) : t;
    return (tl % n) * lpl + tl / n;
  };
  auto site_valid = [&](int m) { return m < n && jj * n + m < T; };

  Vec3<R> c[NS];
  Mat3<R> G = ident<R>();
#pragma unroll
  for (int s = 0; s < NS; ++s) c[s] = vzero<R>();
  bool any = false;
#pragma unroll
  for (int q = 0; q < NM; ++q) {
    const int m = FWD ? q : NM - 1 - q;
    if (!site_valid(m)) continue;
    Mat3<R> U = ldmat(ut_line, tp, link_slot(m));
    if (KEEPU) Uk[KEEPU ? m : 0] = U;
    Mat3<R> A = FWD ? dagger(U) : U;
    if (!any) {
#pragma unroll
      for (int s = 0; s < NS; ++s) c[s] = vscale(inv_mu, v[m][s]);
      G = scale(inv_mu, A);
      any = true;
    } else {
#pragma unroll
      for (int s = 0; s < NS; ++s) c[s] = vscale(inv_mu, matvec_acc(A, c[s], v[m][s]));
      G = scale(inv_mu, matmul(A, G));
    }
  }

  for (int d = 1; d < lpl; d <<= 1) {
    Mat3<R> Gn;
    Vec3<R> cn[NS];
#pragma unroll
    for (int k = 0; k < 9; ++k) Gn.e[k] = FWD ? shfl_up(G.e[k], d, lpl) : shfl_down(G.e[k], d, lpl);
#pragma unroll
    for (int s = 0; s < NS; ++s) cn[s] = FWD ? vshfl_up(c[s], d, lpl) : vshfl_down(c[s], d, lpl);
    const bool has = FWD ? (jj >= d) : (jj + d < lpl);
    if (has) {
#pragma unroll
      for (int s = 0; s < NS; ++s) c[s] = matvec_acc(G, cn[s], c[s]);
      G = matmul(G, Gn);
    }
  }

  const Mat3<R> Lam = ldmat(lam, 1, 0);
  const int root = FWD ? lpl - 1 : 0;
  Vec3<R> wrap[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) wrap[s] = vscale(bc, vshfl_idx(matvec(Lam, c[s]), root, lpl));
  Vec3<R> e[NS];
  {
    Mat3<R> Gn;
    Vec3<R> cn[NS];
#pragma unroll
    for (int k = 0; k < 9; ++k) Gn.e[k] = FWD ? shfl_up(G.e[k], 1, lpl) : shfl_down(G.e[k], 1, lpl);
#pragma unroll
    for (int s = 0; s < NS; ++s) cn[s] = FWD ? vshfl_up(c[s], 1, lpl) : vshfl_down(c[s], 1, lpl);
    const bool edge = FWD ? (jj == 0) : (jj == lpl - 1);
#pragma unroll
    for (int s = 0; s < NS; ++s) e[s] = edge ? wrap[s] : matvec_acc(Gn, wrap[s], cn[s]);
  }

#pragma unroll
  for (int q = 0; q < NM; ++q) {
    const int m = FWD ? q : NM - 1 - q;
    if (!site_valid(m)) continue;
    Mat3<R> U = KEEPU ? Uk[KEEPU ? m : 0] : ldmat(ut_line, tp, link_slot(m));
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Vec3<R> a = FWD ? matvec_dag(U, e[s]) : matvec(U, e[s]);
      e[s] = vscale(inv_mu, vadd(a, v[m][s]));
      v[m][s] = e[s];
    }
  }
}

// ----------------------------------------------------------------------------
// Axial frame: U_0 = 1 except U_0(N_t-1) = P. Lane maps are psi_out = c + a psi_in with a
// scalar a = mu^-(sites); the value entering the top of the line is P s psi(0) (T^-1) and
// the value entering its bottom is P^dag s psi(N_t-1) (T^-dag). Closure: psi(0) = Lambda C_0,
// psi(N_t-1) = Lambda^dag C_last, since (1 - s mu^-N_t P^dag)^-1 = Lambda^dag.
// ----------------------------------------------------------------------------
template <typename R, int NS, bool FWD, int NM>
__device__ __forceinline__ void tline_solve_axial(Vec3<R> (&v)[NM][NS], const Cx<R>* __restrict__ P_line,
                                                  const Cx<R>* __restrict__ lam, const Geom& g, int jj, R inv_mu, R bc) {
  const int T = g.T, lpl = g.lpl, n = g.n;
  auto site_valid = [&](int m) { return m < n && jj * n + m < T; };

  Vec3<R> c[NS];
  R a = R(1);
#pragma unroll
  for (int s = 0; s < NS; ++s) c[s] = vzero<R>();
#pragma unroll
  for (int q = 0; q < NM; ++q) {
    const int m = FWD ? q : NM - 1 - q;
    if (!site_valid(m)) continue;
#pragma unroll
    for (int s = 0; s < NS; ++s) c[s] = vscale(inv_mu, vadd(v[m][s], c[s]));
    a *= inv_mu;
  }

  for (int d = 1; d < lpl; d <<= 1) {
    const R an = FWD ? shfl_up_r(a, d, lpl) : shfl_down_r(a, d, lpl);
    Vec3<R> cn[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) cn[s] = FWD ? vshfl_up(c[s], d, lpl) : vshfl_down(c[s], d, lpl);
    const bool has = FWD ? (jj >= d) : (jj + d < lpl);
    if (has) {
#pragma unroll
      for (int s = 0; s < NS; ++s) c[s] = vaxpy(a, cn[s], c[s]);
      a *= an;
    }
  }

  const int root = FWD ? lpl - 1 : 0;
  Vec3<R> wrap[NS];
  {
    const Mat3<R> Lam = ldmat(lam, 1, 0);
    const Mat3<R> P = ldmat(P_line, 1, 0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      // T^-1 : psi(0) = Lambda C_0, entering value P s psi(0)
      // T^-dag: psi(N_t-1) = Lambda^dag C_last, entering value P^dag s psi(N_t-1)
      Vec3<R> w = FWD ? matvec_dag(P, matvec_dag(Lam, c[s])) : matvec(P, matvec(Lam, c[s]));
      wrap[s] = vscale(bc, vshfl_idx(w, root, lpl));
    }
  }
  Vec3<R> e[NS];
  {
    const R an = FWD ? shfl_up_r(a, 1, lpl) : shfl_down_r(a, 1, lpl);
    const bool edge = FWD ? (jj == 0) : (jj == lpl - 1);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Vec3<R> cn = FWD ? vshfl_up(c[s], 1, lpl) : vshfl_down(c[s], 1, lpl);
      e[s] = edge ? wrap[s] : vaxpy(an, wrap[s], cn);
    }
  }

#pragma unroll
  for (int q = 0; q < NM; ++q) {
    const int m = FWD ? q : NM - 1 - q;
    if (!site_valid(m)) continue;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      e[s] = vscale(inv_mu, vadd(v[m][s], e[s]));
      v[m][s] = e[s];
    }
  }
}

// i sigma_k applied to the two-spin vector (a0, a1): k = 0 (x), 1 (y), 2 (z)
template <typename R>
__device__ __forceinline__ void isigma(int k, const Vec3<R>& a0, const Vec3<R>& a1, Vec3<R>& r0, Vec3<R>& r1) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (k == 0) {
      r0.c[c] = times_i(a1.c[c]);
      r1.c[c] = times_i(a0.c[c]);
    } else if (k == 1) {
      r0.c[c] = a1.c[c];
      r1.c[c] = mk<R>(-a0.c[c].re, -a0.c[c].im);
    } else {
      r0.c[c] = times_i(a0.c[c]);
      r1.c[c] = times_mi(a1.c[c]);
    }
  }
}

// ----------------------------------------------------------------------------
// Spatial hop D_s (§II, Eq. for D_s) at the lane's n sites of line l (parity p):
//   sum_k (1 - gamma_k)/2 U_k(x) psi(x + k) + (1 + gamma_k)/2 U_k^dag(x - k) psi(x - k).
// Dirac-Pauli basis: with psi = (u, d) (upper, lower spin pairs),
//   (1 - gamma_k) psi = (h, -i sigma_k h), h = u + i sigma_k d,
//   (1 + gamma_k) psi = (h, +i sigma_k h), h = u - i sigma_k d,
// so each direction costs two SU(3) matvecs on a half-spinor (App. B: 984 FLOPs/site).
// ----------------------------------------------------------------------------
template <typename R, int NM>
__device__ __forceinline__ void hop_spatial(Vec3<R> (&h)[NM][4], const LineArgs<R>& A, int rhs, int l, int jj) {
  const Geom& g = A.g;
  const int tp = g.tp, Nl = g.Nl, T = g.T, n = g.n;
  int nb[6];
  neighbour_lines(g, A.parity, l, nb);
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int s = 0; s < 4; ++s) h[m][s] = vzero<R>();

#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {  // 0: forward (x + k), 1: backward (x - k)
      const int ln = nb[2 * k + dir];
      const Cx<R>* up = A.src_up + (size_t)(rhs * Nl + ln) * NSPIN_C * tp;
      const Cx<R>* lo = A.src_lo + (size_t)(rhs * Nl + ln) * NSPIN_C * tp;
      constexpr int LNC = SpatialLinkNC<R>::value;
      const Cx<R>* lk = dir == 0 ? A.us_out + (size_t)(k * Nl + l) * LNC * tp
                                 : A.us_nbr + (size_t)(k * Nl + ln) * LNC * tp;
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        if (m >= n || jj * n + m >= T) continue;
        const int sl = m * g.lpl + jj;
        Vec3<R> u0 = ldvec(up, tp, sl), u1 = ldvec(up + 3 * tp, tp, sl);
        Vec3<R> d0 = ldvec(lo, tp, sl), d1 = ldvec(lo + 3 * tp, tp, sl);
        Mat3<R> U = ldlink(lk, tp, sl);
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
        Vec3<R> w0 = dir == 0 ? matvec(U, h0) : matvec_dag(U, h0);
        Vec3<R> w1 = dir == 0 ? matvec(U, h1) : matvec_dag(U, h1);
        h[m][0] = vadd(h[m][0], w0);
        h[m][1] = vadd(h[m][1], w1);
        Vec3<R> r0, r1;
        isigma(k, w0, w1, r0, r1);
        if (dir == 0) {
          h[m][2] = vaxpy(R(-1), r0, h[m][2]);
          h[m][3] = vaxpy(R(-1), r1, h[m][3]);
        } else {
          h[m][2] = vadd(h[m][2], r0);
          h[m][3] = vadd(h[m][3], r1);
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int s = 0; s < 4; ++s) h[m][s] = vscale(R(0.5), h[m][s]);
}

}  // namespace wf
