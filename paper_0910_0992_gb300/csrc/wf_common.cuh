// Device-side building blocks shared by the kernels of libwf: complex numbers,
// SU(3) products, the lattice geometry and the time-line field layout.
//
// Layout ("line-major, lane-interleaved"): a half-lattice field of one 3-D parity
// p3 = (x + y + z) mod 2 holds, for every spatial site of that parity (a "line",
// indexed l = (x >> 1) + (L/2) (y + L z)), the whole time line t = 0 .. T-1.
// Element (rhs, l, c, t) of a field with NC complex components per site sits at
//     ((rhs * Nl + l) * NC + c) * tp + slot(t),   slot(t) = (t % n) * lpl + t / n,
// where a line is processed by lpl lanes of one warp and lane j owns the n
// consecutive times t = n j .. n j + n - 1. Slots with t >= T are padding and are
// kept at zero. With this map a warp instruction that reads component c of the
// m-th site of every lane touches lpl consecutive elements, for the line itself
// and for every spatial neighbour line alike, so both the time-line recurrences
// and the spatial hops load coalesced.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wf_df64.cuh"

namespace wf {

// ----------------------------------------------------------------------------
// Complex arithmetic
// ----------------------------------------------------------------------------
template <typename R>
struct __align__(2 * sizeof(R)) Cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ Cx<R> mk(R a, R b) {
  Cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <typename R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return mk<R>(s * a.re, s * a.im); }
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// acc + a * b
template <typename R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> acc, Cx<R> a, Cx<R> b) {
  return mk<R>(fma(a.re, b.re, fma(-a.im, b.im, acc.re)), fma(a.re, b.im, fma(a.im, b.re, acc.im)));
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ Cx<R> cfmaconj(Cx<R> acc, Cx<R> a, Cx<R> b) {
  return mk<R>(fma(a.re, b.re, fma(a.im, b.im, acc.re)), fma(a.re, b.im, fma(-a.im, b.re, acc.im)));
}
template <typename R>
__device__ __forceinline__ Cx<R> times_i(Cx<R> a) { return mk<R>(-a.im, a.re); }
template <typename R>
__device__ __forceinline__ Cx<R> times_mi(Cx<R> a) { return mk<R>(a.im, -a.re); }
template <typename R>
__device__ __forceinline__ Cx<R> czero() { return mk<R>(R(0), R(0)); }

// one complex element from / to device memory; double-float values live in memory as FP64
template <typename R>
__device__ __forceinline__ Cx<R> ldc(const Cx<R>* p) { return *p; }
template <typename R>
__device__ __forceinline__ void stc(Cx<R>* p, Cx<R> z) { *p = z; }
__device__ __forceinline__ Cx<df64> ldc(const Cx<df64>* p) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  return mk<df64>(df_from_double(v.x), df_from_double(v.y));
}
__device__ __forceinline__ void stc(Cx<df64>* p, Cx<df64> z) {
  *reinterpret_cast<double2*>(p) = make_double2(df_to_double(z.re), df_to_double(z.im));
}

// full-warp shuffles of one real value (float, double or a double-float pair)
template <typename R>
__device__ __forceinline__ R shfl_down_r(R v, int d, int width) { return __shfl_down_sync(0xffffffffu, v, d, width); }
template <typename R>
__device__ __forceinline__ R shfl_up_r(R v, int d, int width) { return __shfl_up_sync(0xffffffffu, v, d, width); }
template <typename R>
__device__ __forceinline__ R shfl_idx_r(R v, int src, int width) { return __shfl_sync(0xffffffffu, v, src, width); }
__device__ __forceinline__ df64 shfl_down_r(df64 v, int d, int width) {
  return df64(__shfl_down_sync(0xffffffffu, v.hi, d, width), __shfl_down_sync(0xffffffffu, v.lo, d, width));
}
__device__ __forceinline__ df64 shfl_up_r(df64 v, int d, int width) {
  return df64(__shfl_up_sync(0xffffffffu, v.hi, d, width), __shfl_up_sync(0xffffffffu, v.lo, d, width));
}
__device__ __forceinline__ df64 shfl_idx_r(df64 v, int src, int width) {
  return df64(__shfl_sync(0xffffffffu, v.hi, src, width), __shfl_sync(0xffffffffu, v.lo, src, width));
}

template <typename R>
__device__ __forceinline__ Cx<R> shfl_down(Cx<R> v, int d, int width) {
  return mk<R>(shfl_down_r(v.re, d, width), shfl_down_r(v.im, d, width));
}
template <typename R>
__device__ __forceinline__ Cx<R> shfl_up(Cx<R> v, int d, int width) {
  return mk<R>(shfl_up_r(v.re, d, width), shfl_up_r(v.im, d, width));
}
template <typename R>
__device__ __forceinline__ Cx<R> shfl_idx(Cx<R> v, int src, int width) {
  return mk<R>(shfl_idx_r(v.re, src, width), shfl_idx_r(v.im, src, width));
}

// ----------------------------------------------------------------------------
// 3x3 colour algebra (row-major 3x3 complex matrices, 3-component vectors)
// ----------------------------------------------------------------------------
template <typename R>
struct Mat3 {
  Cx<R> e[9];
};
template <typename R>
struct Vec3 {
  Cx<R> c[3];
};

template <typename R>
__device__ __forceinline__ Vec3<R> matvec(const Mat3<R>& U, const Vec3<R>& v) {
  Vec3<R> w;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<R> s = cmul(U.e[3 * a + 0], v.c[0]);
    s = cfma(s, U.e[3 * a + 1], v.c[1]);
    w.c[a] = cfma(s, U.e[3 * a + 2], v.c[2]);
  }
  return w;
}
// U^dag v
template <typename R>
__device__ __forceinline__ Vec3<R> matvec_dag(const Mat3<R>& U, const Vec3<R>& v) {
  Vec3<R> w;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<R> s = cfmaconj(czero<R>(), U.e[0 + a], v.c[0]);
    s = cfmaconj(s, U.e[3 + a], v.c[1]);
    w.c[a] = cfmaconj(s, U.e[6 + a], v.c[2]);
  }
  return w;
}
// acc + U v
template <typename R>
__device__ __forceinline__ Vec3<R> matvec_acc(const Mat3<R>& U, const Vec3<R>& v, const Vec3<R>& acc) {
  Vec3<R> w;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<R> s = cfma(acc.c[a], U.e[3 * a + 0], v.c[0]);
    s = cfma(s, U.e[3 * a + 1], v.c[1]);
    w.c[a] = cfma(s, U.e[3 * a + 2], v.c[2]);
  }
  return w;
}
template <typename R>
__device__ __forceinline__ Mat3<R> matmul(const Mat3<R>& A, const Mat3<R>& B) {
  Mat3<R> C;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Cx<R> s = cmul(A.e[3 * a + 0], B.e[0 + b]);
      s = cfma(s, A.e[3 * a + 1], B.e[3 + b]);
      C.e[3 * a + b] = cfma(s, A.e[3 * a + 2], B.e[6 + b]);
    }
  return C;
}
template <typename R>
__device__ __forceinline__ Mat3<R> dagger(const Mat3<R>& A) {
  Mat3<R> C;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) C.e[3 * a + b] = mk<R>(A.e[3 * b + a].re, -A.e[3 * b + a].im);
  return C;
}
template <typename R>
__device__ __forceinline__ Mat3<R> scale(R s, const Mat3<R>& A) {
  Mat3<R> C;
#pragma unroll
  for (int k = 0; k < 9; ++k) C.e[k] = s * A.e[k];
  return C;
}
template <typename R>
__device__ __forceinline__ Mat3<R> ident() {
  Mat3<R> C;
#pragma unroll
  for (int k = 0; k < 9; ++k) C.e[k] = mk<R>(k % 4 == 0 ? R(1) : R(0), R(0));
  return C;
}

// ----------------------------------------------------------------------------
// Geometry
// ----------------------------------------------------------------------------
struct Geom {
  int L, T;
  int Lh;       // L / 2
  int Nl;       // lines per parity: L^3 / 2
  int n;        // time sites per lane
  int lpl;      // lanes per line (power of two, <= 32)
  int tp;       // padded line length n * lpl
  int lpw;      // lines per warp: 32 / lpl
  int by;       // y rows per traversal tile of the line kernels (a divisor of L)
  double mu;    // 1 / (2 kappa_t)
  double gamma_f;
  double bc;    // +1 periodic, -1 antiperiodic in time
};

__host__ __device__ __forceinline__ int slot_of(const Geom& g, int t) { return (t % g.n) * g.lpl + t / g.n; }

// spatial coordinates of line l of parity p
__host__ __device__ __forceinline__ void line_coords(const Geom& g, int p, int l, int& x, int& y, int& z) {
  int xh = l % g.Lh;
  int r = l / g.Lh;
  y = r % g.L;
  z = r / g.L;
  x = 2 * xh + ((y + z + p) & 1);
}
__host__ __device__ __forceinline__ int line_of(const Geom& g, int x, int y, int z) {
  return (x >> 1) + g.Lh * (y + g.L * z);
}
// the 6 spatial neighbour lines (in the other parity): order +x, -x, +y, -y, +z, -z
__host__ __device__ __forceinline__ void neighbour_lines(const Geom& g, int p, int l, int nb[6]) {
  int x, y, z;
  line_coords(g, p, l, x, y, z);
  const int L = g.L;
  nb[0] = line_of(g, (x + 1) % L, y, z);
  nb[1] = line_of(g, (x + L - 1) % L, y, z);
  nb[2] = line_of(g, x, (y + 1) % L, z);
  nb[3] = line_of(g, x, (y + L - 1) % L, z);
  nb[4] = line_of(g, x, y, (z + 1) % L);
  nb[5] = line_of(g, x, y, (z + L - 1) % L);
}

// Spinor component index: spin * 3 + colour. Dirac-Pauli basis: spins 0, 1 are the
// P_+ = (1 + gamma_t)/2 ("upper") half, spins 2, 3 the P_- ("lower") half.
constexpr int NSPIN_C = 12;
constexpr int NLINK_C = 9;

// Spatial links are stored with 9 complex entries in FP64 and with their first two rows only
// (6 entries) in FP32: for an SU(3) matrix the third row is the complex conjugate of the cross
// product of the first two, so the FP32 kernels rebuild it instead of reading it.
template <typename R>
struct SpatialLinkNC {
  static constexpr int value = 9;
};
#ifndef WF_F32_LINK_NC
#define WF_F32_LINK_NC 6
#endif
template <>
struct SpatialLinkNC<float> {
  static_assert(WF_F32_LINK_NC == 6 || WF_F32_LINK_NC == 9, "FP32 links: 6 (two rows) or 9 entries");
  static constexpr int value = WF_F32_LINK_NC;
};

}  // namespace wf
