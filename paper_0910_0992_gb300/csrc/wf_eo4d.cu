// The standard 4-D even-odd (Schur) Wilson operator, the comparator of the temporal
// preconditioner (§II.B, first display: M-hat_4 = M^oo - M^oe (M^ee)^-1 M^eo, which for Wilson
// fermions is mu - mu^-1 D_w^oe D_w^eo with D_w = D_t + D_s / gamma_f; App. B, Wilson case).
//
// Layout of a field of one 4-D parity p4 = (x + y + z + t) mod 2: for every spatial site
// s3 = x + L (y + L z) (all L^3 of them) the T/2 times of that parity,
//     element (rhs, s3, c, h) at ((rhs * L^3 + s3) * 12 + c) * (T/2) + h,   t = 2 h + t0,
// t0 = (p4 + p3(s3)) mod 2. A spatial neighbour (same t, other p4) sits at the same h; a
// temporal neighbour sits at h or h +- 1 of the same spatial site. One thread computes one
// site; consecutive threads take consecutive h, so every load is coalesced. The sources of one
// spatial site run in consecutive CTAs (they share the site's links).
// Links are the handle's (same frame as the temporal preconditioner: in the axial frame
// U_t = 1 except the boundary link P), read through the line layout's index maps.
#include <cstring>
#include <type_traits>

#include "wf_internal.h"
#include "wf_line.cuh"

namespace wf {

constexpr int kEoThreads = 128;
// resident CTAs per SM the dslash is compiled for (4: 128 registers; measured on GB300 1.36x
// faster than 1, and ahead of 6 and 8, which spill)
#ifndef WF_EO_MINB
#define WF_EO_MINB 4
#endif


__device__ __forceinline__ int eo_t0(int par, int x, int y, int z) { return (par + x + y + z) & 1; }

template <typename R, bool AX>
__global__ void __launch_bounds__(kEoThreads, WF_EO_MINB) k_dslash4(const EoArgs<R> A) {
  const Geom& g = A.g;
  const int Th = g.T / 2;
  const int L = g.L;
  const size_t V3 = (size_t)L * L * L;
  const size_t total = (size_t)A.nrhs * V3 * Th;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const bool active = i < total;
  const size_t ii = active ? i : 0;
  // (site position, source, h) with the sources of a site side by side, so that the CTAs of one
  // site's sources run together and share its links through L2; the site positions follow the
  // tiled traversal of the line kernels (all x by g.by rows of y, streamed along z), so that a
  // neighbour's spinor is read again while still in L2
  const int h = (int)(ii % Th);
  const size_t sline = ii / Th;
  const int rhs = (int)(sline % A.nrhs);
  const int pos = (int)(sline / A.nrhs);
  const int x = pos % L;
  int u = pos / L;
  const int yy = u % g.by;
  u /= g.by;
  const int z = u % L, y = (u / L) * g.by + yy;
  const size_t s3 = (size_t)x + L * ((size_t)y + L * z);
  const int p3 = (x + y + z) & 1;
  const int t0 = eo_t0(A.par, x, y, z);
  const int t = 2 * h + t0;
  const int tp = g.tp;
  const int sl = slot_of(g, t);
  const int l = line_of(g, x, y, z);
  const size_t fstride = (size_t)NSPIN_C * Th;  // one site-line of a field
  const int cu = A.swap_in ? 6 : 0, cl = A.swap_in ? 0 : 6;  // component offsets of the halves read

  Vec3<R> acc[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) acc[s] = vzero<R>();

  // spatial hops (same t, same h), scaled by 1 / gamma_f at the end
  const int nbx[6] = {(x + 1) % L, (x + L - 1) % L, x, x, x, x};
  const int nby[6] = {y, y, (y + 1) % L, (y + L - 1) % L, y, y};
  const int nbz[6] = {z, z, z, z, (z + 1) % L, (z + L - 1) % L};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const int d = 2 * k + dir;
      const size_t s3n = (size_t)nbx[d] + L * ((size_t)nby[d] + L * nbz[d]);
      const Cx<R>* nb = A.in + ((size_t)rhs * V3 + s3n) * fstride;
      Vec3<R> u0 = ldvec(nb + cu * Th, Th, h), u1 = ldvec(nb + (cu + 3) * Th, Th, h);
      Vec3<R> d0 = ldvec(nb + cl * Th, Th, h), d1 = ldvec(nb + (cl + 3) * Th, Th, h);
      constexpr int LNC = SpatialLinkNC<R>::value;
      const Cx<R>* lk = dir == 0 ? A.us[p3] + ((size_t)k * g.Nl + l) * LNC * tp
                                 : A.us[1 - p3] + ((size_t)k * g.Nl + line_of(g, nbx[d], nby[d], nbz[d])) * LNC * tp;
      const Mat3<R> U = ldlink(lk, tp, sl);
      Vec3<R> s0, s1;
      isigma(k, d0, d1, s0, s1);
      Vec3<R> h0, h1;  // the projectors' factor 1/2 joins 1 / gamma_f below (exact)
      if (dir == 0) {
        h0 = vadd(u0, s0);
        h1 = vadd(u1, s1);
      } else {
        h0 = vaxpy(R(-1), s0, u0);
        h1 = vaxpy(R(-1), s1, u1);
      }
      Vec3<R> w0 = dir == 0 ? matvec(U, h0) : matvec_dag(U, h0);
      Vec3<R> w1 = dir == 0 ? matvec(U, h1) : matvec_dag(U, h1);
      acc[0] = vadd(acc[0], w0);
      acc[1] = vadd(acc[1], w1);
      Vec3<R> r0, r1;
      isigma(k, w0, w1, r0, r1);
      if (dir == 0) {
        acc[2] = vaxpy(R(-1), r0, acc[2]);
        acc[3] = vaxpy(R(-1), r1, acc[3]);
      } else {
        acc[2] = vadd(acc[2], r0);
        acc[3] = vadd(acc[3], r1);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) acc[s] = vscale(R(0.5) * A.inv_gf, acc[s]);

  // temporal hops: P_- U_t(t) psi(t+1) on spins 2-3, P_+ U_t^dag(t-1) psi(t-1) on spins 0-1
  {
    const Cx<R>* own = A.in + ((size_t)rhs * V3 + s3) * fstride;
    const int hf = (t == g.T - 1) ? 0 : (t + 1) / 2;      // other-parity index of t + 1
    const int hb = (t == 0) ? Th - 1 : (t - 1) / 2;       // other-parity index of t - 1
    const R sf = t == g.T - 1 ? A.bc : R(1), sb = t == 0 ? A.bc : R(1);
    Vec3<R> f0 = ldvec(own + cl * Th, Th, hf), f1 = ldvec(own + (cl + 3) * Th, Th, hf);
    Vec3<R> b0 = ldvec(own + cu * Th, Th, hb), b1 = ldvec(own + (cu + 3) * Th, Th, hb);
    if (AX) {
      if (t == g.T - 1) {
        const Mat3<R> P = ldmat(A.pl[p3] + (size_t)l * 9, 1, 0);
        f0 = matvec(P, f0);
        f1 = matvec(P, f1);
      }
      if (t == 0) {
        const Mat3<R> P = ldmat(A.pl[p3] + (size_t)l * 9, 1, 0);
        b0 = matvec_dag(P, b0);
        b1 = matvec_dag(P, b1);
      }
    } else {
      const Cx<R>* ul = A.ut[p3] + (size_t)l * NLINK_C * tp;
      const Mat3<R> Uf = ldmat(ul, tp, sl);
      const Mat3<R> Ub = ldmat(ul, tp, slot_of(g, t == 0 ? g.T - 1 : t - 1));
      f0 = matvec(Uf, f0);
      f1 = matvec(Uf, f1);
      b0 = matvec_dag(Ub, b0);
      b1 = matvec_dag(Ub, b1);
    }
    acc[0] = vaxpy(sb, b0, acc[0]);
    acc[1] = vaxpy(sb, b1, acc[1]);
    acc[2] = vaxpy(sf, f0, acc[2]);
    acc[3] = vaxpy(sf, f1, acc[3]);
  }

  R nrm = R(0);
  if (active) {
    Cx<R>* o = A.out + ((size_t)rhs * V3 + s3) * fstride;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int so = A.swap_out ? (s + 2) % 4 : s;  // result spin s goes to slot so
      Vec3<R> val = vscale(A.a, acc[s]);
      if (A.x1) val = vaxpy(A.b1, ldvec_stream(A.x1 + ((size_t)rhs * V3 + s3) * fstride + so * 3 * Th, Th, h), val);
      if (A.x2) val = vaxpy(A.b2, ldvec_stream(A.x2 + ((size_t)rhs * V3 + s3) * fstride + so * 3 * Th, Th, h), val);
      if (A.stream_out)
        stvec_stream(o + so * 3 * Th, Th, h, val);
      else
        stvec(o + so * 3 * Th, Th, h, val);
      if (A.norm2) nrm += vnorm2(val);
    }
  }
  if (A.norm2) {
    // |out|^2 per right-hand side: a segmented sum over the warp's lanes. A (site, source) pair
    // holds T/2 consecutive threads, so with T/2 not a multiple of 32 a warp straddles several
    // pairs; each pair's lanes are contiguous and its last lane adds the pair's sum (one atomic per
    // pair and warp instead of one per thread)
    const int lane = threadIdx.x & 31;
    const int key = active ? (int)sline : -1;
    double dn = (double)nrm;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double v = __shfl_up_sync(0xffffffffu, dn, off);
      const int kv = __shfl_up_sync(0xffffffffu, key, off);
      if (lane >= off && kv == key) dn += v;
    }
    const int knext = __shfl_down_sync(0xffffffffu, key, 1);
    if (active && (lane == 31 || knext != key)) atomicAdd(A.norm2 + rhs, dn);
  }
}

template <typename R>
static void launch_dslash4_impl(const EoArgs<R>& a, bool axial, cudaStream_t s) {
  const size_t total = (size_t)a.nrhs * a.g.L * a.g.L * a.g.L * (a.g.T / 2);
  const int blocks = (int)((total + kEoThreads - 1) / kEoThreads);
  if (axial)
    k_dslash4<R, true><<<blocks, kEoThreads, 0, s>>>(a);
  else
    k_dslash4<R, false><<<blocks, kEoThreads, 0, s>>>(a);
  WF_CUDA(cudaGetLastError());
}

// double-float arguments over the same FP64 arrays (see wf_df64.cuh)
static EoArgs<df64> eo_args_df(const EoArgs<double>& a) {
  auto cv = [](const Cx<double>* p) { return reinterpret_cast<const Cx<df64>*>(p); };
  EoArgs<df64> b;
  std::memset(&b, 0, sizeof(b));  // every field defined, including ones added later
  b.g = a.g;
  b.par = a.par;
  b.nrhs = a.nrhs;
  b.in = cv(a.in);
  b.x1 = cv(a.x1);
  b.b1 = df64(a.b1);
  b.x2 = cv(a.x2);
  b.b2 = df64(a.b2);
  b.a = df64(a.a);
  b.swap_in = a.swap_in;
  b.swap_out = a.swap_out;
  b.stream_out = a.stream_out;
  b.df = 0;
  b.out = reinterpret_cast<Cx<df64>*>(a.out);
  b.norm2 = a.norm2;
  for (int p = 0; p < 2; ++p) {
    b.ut[p] = cv(a.ut[p]);
    b.pl[p] = cv(a.pl[p]);
    b.us[p] = cv(a.us[p]);
  }
  b.inv_gf = df64(a.inv_gf);
  b.bc = df64(a.bc);
  return b;
}

template <typename R>
void launch_dslash4(const EoArgs<R>& a, bool axial, cudaStream_t s) {
  if constexpr (std::is_same<R, double>::value) {
    if (a.df) {
      launch_dslash4_impl<df64>(eo_args_df(a), axial, s);
      return;
    }
  }
  launch_dslash4_impl<R>(a, axial, s);
}
template void launch_dslash4<float>(const EoArgs<float>&, bool, cudaStream_t);
template void launch_dslash4<double>(const EoArgs<double>&, bool, cudaStream_t);

// ----------------------------------------------------------------------------
// Conversions: lexicographic complex128 <-> 4-D parity fields (with the frame rotation g of the
// line layout, [l][9][tp] per 3-D parity, or none)
// ----------------------------------------------------------------------------
template <typename R>
__global__ void k_import_eo(const Geom g, const Cx<double>* __restrict__ lex, Cx<R>* even, Cx<R>* odd, int nrhs,
                            const Cx<double>* g0, const Cx<double>* g1, int compact_par) {
  // compact_par < 0: lex is a full field [rhs][t][z][y][x][12]; else lex holds only the sites of
  // 4-D parity compact_par in lexicographic order, [rhs][V/2][12]
  const int L = g.L, Th = g.T / 2;
  const size_t V3 = (size_t)L * L * L, V = V3 * g.T;
  const size_t nsite = compact_par < 0 ? V : V / 2;
  const size_t total = (size_t)nrhs * nsite * 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int sp = (int)(i % 4);
    const size_t k = (i / 4) % nsite;
    const int rhs = (int)(i / (4 * nsite));
    size_t site = compact_par < 0 ? k : 0;
    int x, y, z, t;
    if (compact_par < 0) {
      x = (int)(site % L);
      y = (int)((site / L) % L);
      z = (int)((site / ((size_t)L * L)) % L);
      t = (int)(site / V3);
    } else {
      // k = (t L^3 + z L^2 + y L + x) / 2 with (x + y + z + t) = compact_par mod 2
      const size_t row = k / (L / 2);
      const int xh = (int)(k % (L / 2));
      y = (int)(row % L);
      z = (int)((row / L) % L);
      t = (int)(row / ((size_t)L * L));
      x = 2 * xh + ((compact_par + y + z + t) & 1);
    }
    const int par = (x + y + z + t) & 1;
    Cx<R>* dst = par ? odd : even;
    if (!dst) continue;
    const Cx<double>* src = lex + ((size_t)rhs * nsite + k) * NSPIN_C + sp * 3;
    Cx<double> v[3] = {src[0], src[1], src[2]};
    const int p3 = (x + y + z) & 1;
    const Cx<double>* gr = p3 ? g1 : g0;
    if (gr) {
      const int l = line_of(g, x, y, z), sl = slot_of(g, t);
      Mat3<double> G = ldmat(gr + (size_t)l * 9 * g.tp, g.tp, sl);
      Vec3<double> a;
      for (int c = 0; c < 3; ++c) a.c[c] = v[c];
      a = matvec(G, a);
      for (int c = 0; c < 3; ++c) v[c] = a.c[c];
    }
    const size_t s3 = (size_t)x + L * ((size_t)y + L * z);
    Cx<R>* o = dst + ((size_t)rhs * V3 + s3) * NSPIN_C * Th + sp * 3 * Th + t / 2;
    for (int c = 0; c < 3; ++c) o[c * Th] = mk<R>((R)v[c].re, (R)v[c].im);
  }
}

template <typename R>
__global__ void k_export_eo(const Geom g, const Cx<R>* even, const Cx<R>* odd, Cx<double>* __restrict__ lex, int nrhs,
                            const Cx<double>* g0, const Cx<double>* g1, int compact_par) {
  const int L = g.L, Th = g.T / 2;
  const size_t V3 = (size_t)L * L * L, V = V3 * g.T;
  const size_t nsite = compact_par < 0 ? V : V / 2;
  const size_t total = (size_t)nrhs * nsite * 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int sp = (int)(i % 4);
    const size_t k = (i / 4) % nsite;
    const int rhs = (int)(i / (4 * nsite));
    int x, y, z, t;
    if (compact_par < 0) {
      x = (int)(k % L);
      y = (int)((k / L) % L);
      z = (int)((k / ((size_t)L * L)) % L);
      t = (int)(k / V3);
    } else {
      const size_t row = k / (L / 2);
      const int xh = (int)(k % (L / 2));
      y = (int)(row % L);
      z = (int)((row / L) % L);
      t = (int)(row / ((size_t)L * L));
      x = 2 * xh + ((compact_par + y + z + t) & 1);
    }
    const int par = (x + y + z + t) & 1;
    const Cx<R>* srcf = par ? odd : even;
    const size_t s3 = (size_t)x + L * ((size_t)y + L * z);
    Cx<double> v[3];
    for (int c = 0; c < 3; ++c) {
      v[c] = mk<double>(0.0, 0.0);
      if (srcf) {
        Cx<R> w = srcf[((size_t)rhs * V3 + s3) * NSPIN_C * Th + (sp * 3 + c) * Th + t / 2];
        v[c] = mk<double>((double)w.re, (double)w.im);
      }
    }
    const int p3 = (x + y + z) & 1;
    const Cx<double>* gr = p3 ? g1 : g0;
    if (gr && srcf) {
      const int l = line_of(g, x, y, z), sl = slot_of(g, t);
      Mat3<double> G = ldmat(gr + (size_t)l * 9 * g.tp, g.tp, sl);
      Vec3<double> a;
      for (int c = 0; c < 3; ++c) a.c[c] = v[c];
      a = matvec_dag(G, a);
      for (int c = 0; c < 3; ++c) v[c] = a.c[c];
    }
    Cx<double>* dst = lex + ((size_t)rhs * nsite + k) * NSPIN_C + sp * 3;
    for (int c = 0; c < 3; ++c) dst[c] = v[c];
  }
}

static int eo_grid(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

template <typename R>
void launch_import_eo(const Geom& g, const Cx<double>* lex, Cx<R>* even, Cx<R>* odd, int nrhs, const Cx<double>* g0,
                      const Cx<double>* g1, int compact_par, cudaStream_t s) {
  size_t n = (size_t)nrhs * g.L * g.L * g.L * g.T * 4;
  k_import_eo<R><<<eo_grid(n), 256, 0, s>>>(g, lex, even, odd, nrhs, g0, g1, compact_par);
  WF_CUDA(cudaGetLastError());
}
template <typename R>
void launch_export_eo(const Geom& g, const Cx<R>* even, const Cx<R>* odd, Cx<double>* lex, int nrhs,
                      const Cx<double>* g0, const Cx<double>* g1, int compact_par, cudaStream_t s) {
  size_t n = (size_t)nrhs * g.L * g.L * g.L * g.T * 4;
  k_export_eo<R><<<eo_grid(n), 256, 0, s>>>(g, even, odd, lex, nrhs, g0, g1, compact_par);
  WF_CUDA(cudaGetLastError());
}
template void launch_import_eo<float>(const Geom&, const Cx<double>*, Cx<float>*, Cx<float>*, int, const Cx<double>*,
                                      const Cx<double>*, int, cudaStream_t);
template void launch_import_eo<double>(const Geom&, const Cx<double>*, Cx<double>*, Cx<double>*, int,
                                       const Cx<double>*, const Cx<double>*, int, cudaStream_t);
template void launch_export_eo<float>(const Geom&, const Cx<float>*, const Cx<float>*, Cx<double>*, int,
                                      const Cx<double>*, const Cx<double>*, int, cudaStream_t);
template void launch_export_eo<double>(const Geom&, const Cx<double>*, const Cx<double>*, Cx<double>*, int,
                                       const Cx<double>*, const Cx<double>*, int, cudaStream_t);

}  // namespace wf
