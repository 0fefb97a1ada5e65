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

// gamma_5 = -[[0, 1], [1, 0]] in the Dirac-Pauli basis: component c <- -(component c +- 6)
template <typename R>
__global__ void k_import_spinor(const Geom g, const Cx<double>* __restrict__ lex, Cx<R>* even, Cx<R>* odd, int nrhs,
                                int g5) {
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const size_t total = (size_t)nrhs * V * NSPIN_C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % NSPIN_C);
    const size_t site = (i / NSPIN_C) % V;
    const int rhs = (int)(i / (NSPIN_C * V));
    int x, y, z, t;
    site_coords(g, site, x, y, z, t);
    const int p = (x + y + z) & 1;
    Cx<R>* dst = p ? odd : even;
    if (!dst) continue;
    Cx<double> val;
    if (g5) {
      val = lex[i - c + (c + 6) % 12];
      val.re = -val.re;
      val.im = -val.im;
    } else {
      val = lex[i];
    }
    const int l = line_of(g, x, y, z);
    dst[((size_t)(rhs * g.Nl + l) * NSPIN_C + c) * g.tp + slot_of(g, t)] = mk<R>((R)val.re, (R)val.im);
  }
}

template <typename R>
__global__ void k_export_spinor(const Geom g, const Cx<R>* even, const Cx<R>* odd, Cx<double>* __restrict__ lex,
                                int nrhs, int g5) {
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const size_t total = (size_t)nrhs * V * NSPIN_C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % NSPIN_C);
    const size_t site = (i / NSPIN_C) % V;
    const int rhs = (int)(i / (NSPIN_C * V));
    int x, y, z, t;
    site_coords(g, site, x, y, z, t);
    const int p = (x + y + z) & 1;
    const Cx<R>* src = p ? odd : even;
    const int cs = g5 ? (c + 6) % 12 : c;
    const int l = line_of(g, x, y, z);
    Cx<double> val = mk<double>(0.0, 0.0);
    if (src) {
      Cx<R> v = src[((size_t)(rhs * g.Nl + l) * NSPIN_C + cs) * g.tp + slot_of(g, t)];
      val = mk<double>((double)v.re, (double)v.im);
      if (g5) val = mk<double>(-val.re, -val.im);
    }
    lex[i] = val;
  }
}

// compact half-lattice array of one parity: [rhs][t][l][12] (sites in lexicographic order)
template <typename R>
__global__ void k_import_compact(const Geom g, const Cx<double>* __restrict__ cmp, Cx<R>* half, int nrhs, int g5) {
  const size_t total = (size_t)nrhs * g.T * g.Nl * NSPIN_C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % NSPIN_C);
    const size_t k = i / NSPIN_C;
    const int l = (int)(k % g.Nl);
    const int t = (int)((k / g.Nl) % g.T);
    const int rhs = (int)(k / ((size_t)g.Nl * g.T));
    Cx<double> val;
    if (g5) {
      val = cmp[i - c + (c + 6) % 12];
      val = mk<double>(-val.re, -val.im);
    } else {
      val = cmp[i];
    }
    half[((size_t)(rhs * g.Nl + l) * NSPIN_C + c) * g.tp + slot_of(g, t)] = mk<R>((R)val.re, (R)val.im);
  }
}

template <typename R>
__global__ void k_export_compact(const Geom g, const Cx<R>* half, Cx<double>* __restrict__ cmp, int nrhs, int g5) {
  const size_t total = (size_t)nrhs * g.T * g.Nl * NSPIN_C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % NSPIN_C);
    const size_t k = i / NSPIN_C;
    const int l = (int)(k % g.Nl);
    const int t = (int)((k / g.Nl) % g.T);
    const int rhs = (int)(k / ((size_t)g.Nl * g.T));
    const int cs = g5 ? (c + 6) % 12 : c;
    Cx<R> v = half[((size_t)(rhs * g.Nl + l) * NSPIN_C + cs) * g.tp + slot_of(g, t)];
    Cx<double> val = mk<double>((double)v.re, (double)v.im);
    if (g5) val = mk<double>(-val.re, -val.im);
    cmp[i] = val;
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
                          cudaStream_t s) {
  size_t n = (size_t)nrhs * g.L * g.L * g.L * g.T * NSPIN_C;
  k_import_spinor<R><<<grid_for(n), kThreads, 0, s>>>(g, lex, even, odd, nrhs, g5);
  WF_CUDA(cudaGetLastError());
}
template <typename R>
void launch_export_spinor(const Geom& g, const Cx<R>* even, const Cx<R>* odd, Cx<double>* lex, int nrhs, int g5,
                          cudaStream_t s) {
  size_t n = (size_t)nrhs * g.L * g.L * g.L * g.T * NSPIN_C;
  k_export_spinor<R><<<grid_for(n), kThreads, 0, s>>>(g, even, odd, lex, nrhs, g5);
  WF_CUDA(cudaGetLastError());
}
template <typename R>
void launch_import_compact(const Geom& g, const Cx<double>* cmp, Cx<R>* half, int nrhs, int g5, cudaStream_t s) {
  size_t n = (size_t)nrhs * g.T * g.Nl * NSPIN_C;
  k_import_compact<R><<<grid_for(n), kThreads, 0, s>>>(g, cmp, half, nrhs, g5);
  WF_CUDA(cudaGetLastError());
}
template <typename R>
void launch_export_compact(const Geom& g, const Cx<R>* half, Cx<double>* cmp, int nrhs, int g5, cudaStream_t s) {
  size_t n = (size_t)nrhs * g.T * g.Nl * NSPIN_C;
  k_export_compact<R><<<grid_for(n), kThreads, 0, s>>>(g, half, cmp, nrhs, g5);
  WF_CUDA(cudaGetLastError());
}
#define WF_INST(R)                                                                                             \
  template void launch_import_spinor<R>(const Geom&, const Cx<double>*, Cx<R>*, Cx<R>*, int, int, cudaStream_t); \
  template void launch_export_spinor<R>(const Geom&, const Cx<R>*, const Cx<R>*, Cx<double>*, int, int,         \
                                        cudaStream_t);                                                         \
  template void launch_import_compact<R>(const Geom&, const Cx<double>*, Cx<R>*, int, int, cudaStream_t);      \
  template void launch_export_compact<R>(const Geom&, const Cx<R>*, Cx<double>*, int, int, cudaStream_t);
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

void launch_d2f(const Cx<double>* in, Cx<float>* out, size_t n, cudaStream_t s) {
  k_d2f<<<grid_for(n), kThreads, 0, s>>>(in, out, n);
  WF_CUDA(cudaGetLastError());
}
void launch_f2d(const Cx<float>* in, Cx<double>* out, size_t n, cudaStream_t s) {
  k_f2d<<<grid_for(n), kThreads, 0, s>>>(in, out, n);
  WF_CUDA(cudaGetLastError());
}

}  // namespace wf
