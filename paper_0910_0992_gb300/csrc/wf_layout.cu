// Layout conversions between the C-ABI's lexicographic complex128 arrays and the
// internal line layout, gauge ingest, and the per-line wrap-around matrices Lambda.
#include "wf_internal.h"

namespace wf {

constexpr int kThreads = 256;

static inline int nblocks(size_t n, int threads = kThreads) {
  size_t b = (n + threads - 1) / threads;
  return (int)(b > 0x7fffffff ? 0x7fffffff : b);
}

// site index (t, z, y, x) lexicographic with x fastest
__device__ __forceinline__ void site_coords(const Geom& g, size_t site, int& x, int& y, int& z, int& t) {
  x = (int)(site % g.L);
  size_t r = site / g.L;
  y = (int)(r % g.L);
  r /= g.L;
  z = (int)(r % g.L);
  t = (int)(r / g.L);
}

// gamma_5 = -[[0, 1], [1, 0]] in the Dirac-Pauli basis: spin s <- -(spin s +- 2).
// Optional colour rotation per site (axial frame): import psi' = g psi, export psi = g^dag psi'.
// g (if not null) is given per parity as [l][9][tp] in FP64.
__device__ __forceinline__ void rotate3(const Cx<double>* __restrict__ gl, int tp, int sl, bool dag, Cx<double> (&v)[3]) {
  Mat3<double> G;
#pragma unroll
  for (int k = 0; k < 9; ++k) G.e[k] = gl[k * tp + sl];
  Vec3<double> x;
#pragma unroll
  for (int k = 0; k < 3; ++k) x.c[k] = v[k];
  Vec3<double> y = dag ? matvec_dag(G, x) : matvec(G, x);
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = y.c[k];
}

// One thread per (rhs, parity, line, slot): all four spins of the site, so that the stores (import)
// and loads (export) of the line layout are coalesced over the slots, the rotation g is loaded
// once per site, and the lexicographic side moves each site's 192 contiguous bytes. Padding
// slots (t >= T) are written as zero on import.
__device__ __forceinline__ int slot_time(const Geom& g, int sl) { return (sl % g.lpl) * g.n + sl / g.lpl; }

template <typename R>
__global__ void k_import_spinor(const Geom g, const Cx<double>* __restrict__ lex, Cx<R>* even, Cx<R>* odd, int nrhs,
                                int g5, const Cx<double>* g_e, const Cx<double>* g_o) {
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const size_t per_p = (size_t)g.Nl * g.tp;
  const size_t total = (size_t)nrhs * 2 * per_p;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int sl = (int)(i % g.tp);
    const int l = (int)((i / g.tp) % g.Nl);
    const int p = (int)((i / per_p) % 2);
    const int rhs = (int)(i / (2 * per_p));
    Cx<R>* dst = p ? odd : even;
    if (!dst) continue;
    Cx<R>* out = dst + (size_t)(rhs * g.Nl + l) * NSPIN_C * g.tp + sl;
    const int t = slot_time(g, sl);
    if (t >= g.T) {
#pragma unroll
      for (int k = 0; k < NSPIN_C; ++k) out[(size_t)k * g.tp] = mk<R>(R(0), R(0));
      continue;
    }
    int x, y, z;
    line_coords(g, p, l, x, y, z);
    const size_t site = (size_t)x + g.L * ((size_t)y + g.L * ((size_t)z + (size_t)g.L * t));
    const Cx<double>* src = lex + ((size_t)rhs * V + site) * NSPIN_C;
    const Cx<double>* gr = p ? g_o : g_e;
    Mat3<double> G;
    if (gr) {
#pragma unroll
      for (int k = 0; k < 9; ++k) G.e[k] = gr[((size_t)l * 9 + k) * g.tp + sl];
    }
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
      const int ssrc = g5 ? (sp + 2) % 4 : sp;
      Vec3<double> v;
#pragma unroll
      for (int c = 0; c < 3; ++c) v.c[c] = g5 ? mk<double>(-src[ssrc * 3 + c].re, -src[ssrc * 3 + c].im) : src[ssrc * 3 + c];
      if (gr) v = matvec(G, v);
#pragma unroll
      for (int c = 0; c < 3; ++c) out[(size_t)(sp * 3 + c) * g.tp] = mk<R>((R)v.c[c].re, (R)v.c[c].im);
    }
  }
}

template <typename R>
__global__ void k_export_spinor(const Geom g, const Cx<R>* even, const Cx<R>* odd, Cx<double>* __restrict__ lex,
                                int nrhs, int g5, const Cx<double>* g_e, const Cx<double>* g_o) {
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const size_t per_p = (size_t)g.Nl * g.tp;
  const size_t total = (size_t)nrhs * 2 * per_p;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int sl = (int)(i % g.tp);
    const int l = (int)((i / g.tp) % g.Nl);
    const int p = (int)((i / per_p) % 2);
    const int rhs = (int)(i / (2 * per_p));
    const int t = slot_time(g, sl);
    if (t >= g.T) continue;
    int x, y, z;
    line_coords(g, p, l, x, y, z);
    const size_t site = (size_t)x + g.L * ((size_t)y + g.L * ((size_t)z + (size_t)g.L * t));
    Cx<double>* dst = lex + ((size_t)rhs * V + site) * NSPIN_C;
    const Cx<R>* src = p ? odd : even;
    if (!src) {
#pragma unroll
      for (int k = 0; k < NSPIN_C; ++k) dst[k] = mk<double>(0.0, 0.0);
      continue;
    }
    const Cx<R>* in = src + (size_t)(rhs * g.Nl + l) * NSPIN_C * g.tp + sl;
    const Cx<double>* gr = p ? g_o : g_e;
    Mat3<double> G;
    if (gr) {
#pragma unroll
      for (int k = 0; k < 9; ++k) G.e[k] = gr[((size_t)l * 9 + k) * g.tp + sl];
    }
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
      const int ss = g5 ? (sp + 2) % 4 : sp;
      Vec3<double> v;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const Cx<R> w = in[(size_t)(ss * 3 + c) * g.tp];
        v.c[c] = mk<double>((double)w.re, (double)w.im);
      }
      if (gr) v = matvec_dag(G, v);
#pragma unroll
      for (int c = 0; c < 3; ++c) dst[sp * 3 + c] = g5 ? mk<double>(-v.c[c].re, -v.c[c].im) : v.c[c];
    }
  }
}

// compact half-lattice array of one parity: [rhs][t][l][12] (sites in lexicographic order)
template <typename R>
__global__ void k_import_compact(const Geom g, const Cx<double>* __restrict__ cmp, Cx<R>* half, int nrhs, int g5,
                                 const Cx<double>* gr) {
  const size_t total = (size_t)nrhs * g.T * g.Nl * 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int sp = (int)(i % 4);
    const size_t k = i / 4;
    const int l = (int)(k % g.Nl);
    const int t = (int)((k / g.Nl) % g.T);
    const int rhs = (int)(k / ((size_t)g.Nl * g.T));
    const int ssrc = g5 ? (sp + 2) % 4 : sp;
    const Cx<double>* src = cmp + k * NSPIN_C + ssrc * 3;
    Cx<double> v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = g5 ? mk<double>(-src[c].re, -src[c].im) : src[c];
    const int sl = slot_of(g, t);
    if (gr) rotate3(gr + (size_t)l * 9 * g.tp, g.tp, sl, false, v);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      half[((size_t)(rhs * g.Nl + l) * NSPIN_C + sp * 3 + c) * g.tp + sl] = mk<R>((R)v[c].re, (R)v[c].im);
  }
}

template <typename R>
__global__ void k_export_compact(const Geom g, const Cx<R>* half, Cx<double>* __restrict__ cmp, int nrhs, int g5,
                                 const Cx<double>* gr) {
  const size_t total = (size_t)nrhs * g.T * g.Nl * 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int sp = (int)(i % 4);
    const size_t k = i / 4;
    const int l = (int)(k % g.Nl);
    const int t = (int)((k / g.Nl) % g.T);
    const int rhs = (int)(k / ((size_t)g.Nl * g.T));
    const int ss = g5 ? (sp + 2) % 4 : sp;
    const int sl = slot_of(g, t);
    Cx<double> v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cx<R> w = half[((size_t)(rhs * g.Nl + l) * NSPIN_C + ss * 3 + c) * g.tp + sl];
      v[c] = mk<double>((double)w.re, (double)w.im);
    }
    if (gr) rotate3(gr + (size_t)l * 9 * g.tp, g.tp, sl, true, v);
    Cx<double>* dst = cmp + k * NSPIN_C + sp * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) dst[c] = g5 ? mk<double>(-v[c].re, -v[c].im) : v[c];
  }
}

// gauge field U[t][z][y][x][mu][row][col] -> U_t per parity [l][9][tp] and forward
// spatial links per parity [mu][l][9][tp]
__global__ void k_import_gauge(const Geom g, const Cx<double>* __restrict__ lex, Cx<double>* ut0, Cx<double>* ut1,
                               Cx<double>* us0, Cx<double>* us1) {
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const size_t total = V * 4 * 9;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % 9);
    const int mu = (int)((i / 9) % 4);
    const size_t site = i / 36;
    int x, y, z, t;
    site_coords(g, site, x, y, z, t);
    const int p = (x + y + z) & 1;
    const int l = line_of(g, x, y, z);
    const int sl = slot_of(g, t);
    if (mu == 3) {
      Cx<double>* ut = p ? ut1 : ut0;
      ut[((size_t)l * 9 + k) * g.tp + sl] = lex[i];
    } else {
      Cx<double>* us = p ? us1 : us0;
      us[(((size_t)mu * g.Nl + l) * 9 + k) * g.tp + sl] = lex[i];
    }
  }
}

__device__ __forceinline__ Mat3<double> ldmat_d(const Cx<double>* base, int tp, int slot) {
  Mat3<double> U;
#pragma unroll
  for (int k = 0; k < 9; ++k) U.e[k] = base[k * tp + slot];
  return U;
}

// 3x3 inverse by the adjugate; returns |det|
__device__ double inv3(const Mat3<double>& A, Mat3<double>& Ai) {
  const Cx<double>* a = A.e;
  Cx<double> c00 = cmul(a[4], a[8]) - cmul(a[5], a[7]);
  Cx<double> c01 = cmul(a[5], a[6]) - cmul(a[3], a[8]);
  Cx<double> c02 = cmul(a[3], a[7]) - cmul(a[4], a[6]);
  Cx<double> det = cmul(a[0], c00) + cmul(a[1], c01) + cmul(a[2], c02);
  double d2 = det.re * det.re + det.im * det.im;
  Cx<double> id = mk<double>(det.re / d2, -det.im / d2);
  Cx<double> adj[9];
  adj[0] = c00;
  adj[3] = c01;
  adj[6] = c02;
  adj[1] = cmul(a[2], a[7]) - cmul(a[1], a[8]);
  adj[4] = cmul(a[0], a[8]) - cmul(a[2], a[6]);
  adj[7] = cmul(a[1], a[6]) - cmul(a[0], a[7]);
  adj[2] = cmul(a[1], a[5]) - cmul(a[2], a[4]);
  adj[5] = cmul(a[2], a[3]) - cmul(a[0], a[5]);
  adj[8] = cmul(a[0], a[4]) - cmul(a[1], a[3]);
  for (int k = 0; k < 9; ++k) Ai.e[k] = cmul(adj[k], id);
  return sqrt(d2);
}

// Per line: Lambda_b = (I - s mu^-N_t P)^-1, P = U_t(0) U_t(1) ... U_t(N_t-1), closes T^-1;
// Lambda_f = (I - s mu^-N_t Q)^-1, Q = U_t^dag(N_t-2) ... U_t^dag(0) U_t^dag(N_t-1), closes
// T^-dag in the lane-scan formulation (§II.A step 1; X(0) = -s mu^-N_t P).
__global__ void k_tline_init(const Geom g, const Cx<double>* __restrict__ ut, Cx<double>* lamb, Cx<double>* lamf,
                             int* singular) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= g.Nl) return;
  const int T = g.T;
  const Cx<double>* line = ut + (size_t)l * 9 * g.tp;
  Mat3<double> P = ident<double>();
  for (int t = T - 1; t >= 0; --t) P = matmul(ldmat_d(line, g.tp, slot_of(g, t)), P);
  Mat3<double> Q = dagger(ldmat_d(line, g.tp, slot_of(g, T - 1)));
  for (int t = 1; t < T; ++t) Q = matmul(dagger(ldmat_d(line, g.tp, slot_of(g, t - 1))), Q);
  const double f = g.bc * pow(g.mu, -(double)T);
  Mat3<double> Ab, Af, Ib, If;
  for (int k = 0; k < 9; ++k) {
    const double id = (k % 4 == 0) ? 1.0 : 0.0;
    Ab.e[k] = mk<double>(id - f * P.e[k].re, -f * P.e[k].im);
    Af.e[k] = mk<double>(id - f * Q.e[k].re, -f * Q.e[k].im);
  }
  const double db = inv3(Ab, Ib);
  const double df = inv3(Af, If);
  if (!(db > 1e-12) || !(df > 1e-12)) atomicExch(singular, 1);
  for (int k = 0; k < 9; ++k) {
    lamb[(size_t)l * 9 + k] = Ib.e[k];
    lamf[(size_t)l * 9 + k] = If.e[k];
  }
}

// Axial (temporal) frame (§II.C; App. C): per line, g(t) = U_t(0) U_t(1) ... U_t(t-1), g(0) = 1,
// so that U_t'(t) = g(t) U_t(t) g(t+1)^dag = 1 for t < N_t - 1 and U_t'(N_t - 1) = g(N_t - 1) U_t(N_t - 1)
// = P, the Polyakov product. Written in place of U_t (ut becomes g); P,
// Lambda = (1 - s mu^-N_t P)^-1 and the wrap matrix K = P Lambda per line. Lambda is a function
// of P, so K = Lambda P as well and K^dag = Lambda^dag P^dag closes T^-dag.
__global__ void k_axial_frame(const Geom g, Cx<double>* ut_to_g, Cx<double>* pl, Cx<double>* lamb, Cx<double>* wrap,
                              int* singular) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= g.Nl) return;
  Cx<double>* line = ut_to_g + (size_t)l * 9 * g.tp;
  Mat3<double> run = ident<double>();
  for (int t = 0; t < g.T; ++t) {
    const int sl = slot_of(g, t);
    const Mat3<double> u = ldmat_d(line, g.tp, sl);
    for (int k = 0; k < 9; ++k) line[k * g.tp + sl] = run.e[k];
    run = matmul(run, u);
  }
  const double f = g.bc * pow(g.mu, -(double)g.T);
  Mat3<double> A, Ai;
  for (int k = 0; k < 9; ++k) {
    const double id = (k % 4 == 0) ? 1.0 : 0.0;
    A.e[k] = mk<double>(id - f * run.e[k].re, -f * run.e[k].im);
  }
  const double d = inv3(A, Ai);
  if (!(d > 1e-12)) atomicExch(singular, 1);
  const Mat3<double> K = matmul(run, Ai);
  for (int k = 0; k < 9; ++k) {
    pl[(size_t)l * 9 + k] = run.e[k];
    lamb[(size_t)l * 9 + k] = Ai.e[k];
    wrap[(size_t)l * 9 + k] = K.e[k];
  }
}

// spatial links into the axial frame, in place: U_k'(x) = g(x) U_k(x) g(x + k)^dag
__global__ void k_rotate_links(const Geom g, int p, Cx<double>* us_p, const Cx<double>* g_p, const Cx<double>* g_q) {
  const size_t total = (size_t)3 * g.Nl * g.T;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(i % g.T);
    const int l = (int)((i / g.T) % g.Nl);
    const int k = (int)(i / ((size_t)g.T * g.Nl));
    int nb[6];
    neighbour_lines(g, p, l, nb);
    const int sl = slot_of(g, t);
    Cx<double>* U = us_p + ((size_t)k * g.Nl + l) * 9 * g.tp;
    const Mat3<double> gx = ldmat_d(g_p + (size_t)l * 9 * g.tp, g.tp, sl);
    const Mat3<double> gy = ldmat_d(g_q + (size_t)nb[2 * k] * 9 * g.tp, g.tp, sl);
    const Mat3<double> r = matmul(matmul(gx, ldmat_d(U, g.tp, sl)), dagger(gy));
    for (int e = 0; e < 9; ++e) U[e * g.tp + sl] = r.e[e];
  }
}

__global__ void k_d2f(const Cx<double>* __restrict__ in, Cx<float>* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = mk<float>((float)in[i].re, (float)in[i].im);
}
__global__ void k_f2d(const Cx<float>* __restrict__ in, Cx<double>* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = mk<double>((double)in[i].re, (double)in[i].im);
}

static int grid_for(size_t n) {
  int b = nblocks(n);
  return b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b);
}

template <typename R>
void launch_import_spinor(const Geom& g, const Cx<double>* lex, Cx<R>* even, Cx<R>* odd, int nrhs, int g5,
                          const Cx<double>* g_e, const Cx<double>* g_o, cudaStream_t s) {
  const size_t n = (size_t)nrhs * 2 * g.Nl * g.tp;
  k_import_spinor<R><<<grid_for(n), kThreads, 0, s>>>(g, lex, even, odd, nrhs, g5, g_e, g_o);
  WF_CUDA(cudaGetLastError());
}
template <typename R>
void launch_export_spinor(const Geom& g, const Cx<R>* even, const Cx<R>* odd, Cx<double>* lex, int nrhs, int g5,
                          const Cx<double>* g_e, const Cx<double>* g_o, cudaStream_t s) {
  const size_t n = (size_t)nrhs * 2 * g.Nl * g.tp;
  k_export_spinor<R><<<grid_for(n), kThreads, 0, s>>>(g, even, odd, lex, nrhs, g5, g_e, g_o);
  WF_CUDA(cudaGetLastError());
}
template <typename R>
void launch_import_compact(const Geom& g, const Cx<double>* cmp, Cx<R>* half, int nrhs, int g5,
                           const Cx<double>* gr, cudaStream_t s) {
  size_t n = (size_t)nrhs * g.T * g.Nl * 4;
  k_import_compact<R><<<grid_for(n), kThreads, 0, s>>>(g, cmp, half, nrhs, g5, gr);
  WF_CUDA(cudaGetLastError());
}
template <typename R>
void launch_export_compact(const Geom& g, const Cx<R>* half, Cx<double>* cmp, int nrhs, int g5,
                           const Cx<double>* gr, cudaStream_t s) {
  size_t n = (size_t)nrhs * g.T * g.Nl * 4;
  k_export_compact<R><<<grid_for(n), kThreads, 0, s>>>(g, half, cmp, nrhs, g5, gr);
  WF_CUDA(cudaGetLastError());
}
#define WF_INST(R)                                                                                          \
  template void launch_import_spinor<R>(const Geom&, const Cx<double>*, Cx<R>*, Cx<R>*, int, int,             \
                                        const Cx<double>*, const Cx<double>*, cudaStream_t);                \
  template void launch_export_spinor<R>(const Geom&, const Cx<R>*, const Cx<R>*, Cx<double>*, int, int,      \
                                        const Cx<double>*, const Cx<double>*, cudaStream_t);                \
  template void launch_import_compact<R>(const Geom&, const Cx<double>*, Cx<R>*, int, int, const Cx<double>*, \
                                         cudaStream_t);                                                     \
  template void launch_export_compact<R>(const Geom&, const Cx<R>*, Cx<double>*, int, int, const Cx<double>*, \
                                         cudaStream_t);
WF_INST(float)
WF_INST(double)
#undef WF_INST

void launch_import_gauge(const Geom& g, const Cx<double>* lex, Cx<double>* ut[2], Cx<double>* us[2], cudaStream_t s) {
  size_t n = (size_t)g.L * g.L * g.L * g.T * 36;
  k_import_gauge<<<grid_for(n), kThreads, 0, s>>>(g, lex, ut[0], ut[1], us[0], us[1]);
  WF_CUDA(cudaGetLastError());
}

void launch_tline_init(const Geom& g, const Cx<double>* ut, Cx<double>* lamb, Cx<double>* lamf, int* singular,
                       cudaStream_t s) {
  k_tline_init<<<(g.Nl + 127) / 128, 128, 0, s>>>(g, ut, lamb, lamf, singular);
  WF_CUDA(cudaGetLastError());
}

void launch_axial_frame(const Geom& g, Cx<double>* ut_to_g, Cx<double>* pl, Cx<double>* lamb, Cx<double>* wrap,
                        int* singular, cudaStream_t s) {
  k_axial_frame<<<(g.Nl + 127) / 128, 128, 0, s>>>(g, ut_to_g, pl, lamb, wrap, singular);
  WF_CUDA(cudaGetLastError());
}

void launch_rotate_links(const Geom& g, Cx<double>* us[2], const Cx<double>* gg[2], cudaStream_t s) {
  size_t n = (size_t)3 * g.Nl * g.T;
  for (int p = 0; p < 2; ++p) k_rotate_links<<<grid_for(n), kThreads, 0, s>>>(g, p, us[p], gg[p], gg[1 - p]);
  WF_CUDA(cudaGetLastError());
}

// FP32 spatial links: rows 0 and 1 of every FP64 link ([3][Nl][9][tp] -> [3][Nl][6][tp])
__global__ void k_d2f_links(const Cx<double>* __restrict__ in, Cx<float>* __restrict__ out, size_t nlinks, int tp) {
  constexpr int NC = SpatialLinkNC<float>::value;
  const size_t total = nlinks * NC * (size_t)tp;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t sl = i % tp;
    const size_t e = (i / tp) % NC;
    const size_t lk = i / ((size_t)tp * NC);
    const Cx<double> v = in[(lk * 9 + e) * tp + sl];
    out[i] = mk<float>((float)v.re, (float)v.im);
  }
}

void launch_d2f_links(const Cx<double>* in, Cx<float>* out, size_t nlinks, int tp, cudaStream_t s) {
  k_d2f_links<<<grid_for(nlinks * SpatialLinkNC<float>::value * (size_t)tp), kThreads, 0, s>>>(in, out, nlinks, tp);
  WF_CUDA(cudaGetLastError());
}

// Gauge-field check at load: every link must be finite and in SU(3) (the FP32 kernels rebuild a
// link's third row from the first two, which holds only for det U = 1 and U^dag U = 1). One
// thread per link; flag |= 1 for a non-finite entry, |= 2 for max |(U^dag U - 1)_ij| or
// |det U - 1| above tol.
__global__ void k_check_links(const Cx<double>* __restrict__ U, size_t nlinks, double tol, int* flag) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= nlinks) return;
  Mat3<double> A;
  bool finite = true;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    A.e[k] = U[i * 9 + k];
    finite = finite && isfinite(A.e[k].re) && isfinite(A.e[k].im);
  }
  if (!finite) {
    atomicOr(flag, 1);
    return;
  }
  double dev = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Cx<double> s = czero<double>();  // (U^dag U)_ab = sum_c conj(U_ca) U_cb
#pragma unroll
      for (int c = 0; c < 3; ++c) s = cfmaconj(s, A.e[3 * c + a], A.e[3 * c + b]);
      if (a == b) s.re -= 1.0;
      dev = fmax(dev, fmax(fabs(s.re), fabs(s.im)));
    }
  // det U by cofactors along the first row
  const Cx<double>* e = A.e;
  const Cx<double> m0 = cmul(e[4], e[8]) - cmul(e[5], e[7]);
  const Cx<double> m1 = cmul(e[3], e[8]) - cmul(e[5], e[6]);
  const Cx<double> m2 = cmul(e[3], e[7]) - cmul(e[4], e[6]);
  const Cx<double> det = cmul(e[0], m0) - cmul(e[1], m1) + cmul(e[2], m2);
  dev = fmax(dev, fmax(fabs(det.re - 1.0), fabs(det.im)));
  if (!(dev <= tol)) atomicOr(flag, 2);
}

void launch_check_links(const Cx<double>* U, size_t nlinks, double tol, int* flag, cudaStream_t s) {
  const int threads = 256;
  k_check_links<<<(unsigned)((nlinks + threads - 1) / threads), threads, 0, s>>>(U, nlinks, tol, flag);
  WF_CUDA(cudaGetLastError());
}

void launch_d2f(const Cx<double>* in, Cx<float>* out, size_t n, cudaStream_t s) {
  k_d2f<<<grid_for(n), kThreads, 0, s>>>(in, out, n);
  WF_CUDA(cudaGetLastError());
}
void launch_f2d(const Cx<float>* in, Cx<double>* out, size_t n, cudaStream_t s) {
  k_f2d<<<grid_for(n), kThreads, 0, s>>>(in, out, n);
  WF_CUDA(cudaGetLastError());
}

}  // namespace wf
