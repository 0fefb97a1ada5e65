// wf_temporal_logdet: log det(mu - D_t), the determinant of the temporal preconditioner, and
// its force.
//
// C_L^-1 C_R^-1 = P_- T + P_+ T^dag = mu - D_t (§II.A), and C_L M C_R has unit diagonal blocks
// in the 3-D parity split with Schur complement M-hat (§II.B), so det M = det(M-hat)
// det(mu - D_t): a hybrid Monte Carlo run with the preconditioned operator carries this factor
// in its Hamiltonian (§IV). T of one spatial line x is mu on the diagonal, -U_t(t) coupling t to
// t+1 and -s U_t(N_t - 1) across the wrap, so det T(x) = det(mu^N_t 1 - s P(x)) with the ordered
// product P(x) = U_t(0) U_t(1) ... U_t(N_t - 1); each projector holds two spin components, so
//   log det(mu - D_t) = 4 sum_x [3 N_t log mu + log|det(1 - s mu^-N_t P(x))|].
// For U_t(x, t) -> exp(i eps T_a) U_t(x, t), T_a = lambda_a / 2, with A(t) = U_t(0) ... U_t(t-1):
//   d log det(mu - D_t) / d eps = -4 s Re Tr[i T_a Z(t)],   Z(t) = A(t)^dag Z(0) A(t),
//   Z(0) = P (mu^N_t 1 - s P)^-1 = mu^-N_t P (1 - s mu^-N_t P)^-1
// (Z(t) = U_t(t) ... U_t(N_t-1) (mu^N_t - s P)^-1 U_t(0) ... U_t(t-1), and A(t) is unitary).
// In the axial frame the handle stores A(t) as the frame rotation g(t) and P per line; in the
// caller's frame the line kernel forms the prefix products A(t) from U_t.
//
// Kernels (all FP64): k_tdet_line, one thread per spatial line of both parities (P, the 3x3
// determinant and inverse, Z(0)); k_tdet_force, one thread per site in slot order (coalesced
// reads of A(t)), the rotation A^dag Z(0) A and its projection on the eight generators, writing
// the site's 32 force entries (zero for the spatial links); k_tdet_sum, one block adding the
// per-line logarithms in a fixed order (deterministic).
#include <cmath>
#include <cstring>
#include <string>

#include "wf_handle.h"
#include "wf_line.cuh"

using namespace wf;

namespace {

struct DetArgs {
  Geom g;
  int axial;
  const Cx<double>* ut[2];  // axial frame: rotation g(t) = A(t); caller's frame: U_t
  const Cx<double>* pl[2];  // axial frame: P per line [Nl][9]
  Cx<double>* prefix[2];    // caller's frame: A(t), written by k_tdet_line ([Nl][9][tp])
  double c;                 // s mu^-N_t
  double mu_pow;            // mu^-N_t
  double coef;              // -4 s
  double* ld;               // [2 Nl] log|det(1 - s mu^-N_t P)|
  Cx<double>* z0;           // [2 Nl][9] Z(0)
  double* F;                // [t][z][y][x][mu][8]
};

constexpr int kLineBlock = 128;
constexpr int kSiteBlock = 256;
constexpr int kSumBlock = 256;

__device__ __forceinline__ Cx<double> cdet3(const Mat3<double>& A, Cx<double>* cof) {
  const Cx<double>* a = A.e;
  cof[0] = cmul(a[4], a[8]) - cmul(a[5], a[7]);
  cof[1] = cmul(a[5], a[6]) - cmul(a[3], a[8]);
  cof[2] = cmul(a[3], a[7]) - cmul(a[4], a[6]);
  return cmul(a[0], cof[0]) + cmul(a[1], cof[1]) + cmul(a[2], cof[2]);
}

// inverse of a 3x3 complex matrix by its adjugate; returns the determinant
__device__ Cx<double> inverse3(const Mat3<double>& A, Mat3<double>& Ai) {
  const Cx<double>* a = A.e;
  Cx<double> cof[3];
  const Cx<double> det = cdet3(A, cof);
  const double d2 = det.re * det.re + det.im * det.im;
  const Cx<double> id = mk<double>(det.re / d2, -det.im / d2);
  Cx<double> adj[9];
  adj[0] = cof[0];
  adj[3] = cof[1];
  adj[6] = cof[2];
  adj[1] = cmul(a[2], a[7]) - cmul(a[1], a[8]);
  adj[4] = cmul(a[0], a[8]) - cmul(a[2], a[6]);
  adj[7] = cmul(a[1], a[6]) - cmul(a[0], a[7]);
  adj[2] = cmul(a[1], a[5]) - cmul(a[2], a[4]);
  adj[5] = cmul(a[2], a[3]) - cmul(a[0], a[5]);
  adj[8] = cmul(a[0], a[4]) - cmul(a[1], a[3]);
#pragma unroll
  for (int k = 0; k < 9; ++k) Ai.e[k] = cmul(adj[k], id);
  return det;
}

__global__ void __launch_bounds__(kLineBlock) k_tdet_line(const DetArgs A) {
  const Geom& g = A.g;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Nl) return;
  const int p = i / g.Nl;
  const int l = i % g.Nl;
  Mat3<double> P;
  if (A.axial) {
    P = ldmat(A.pl[p] + (size_t)l * 9, 1, 0);
  } else {
    const Cx<double>* u = A.ut[p] + (size_t)l * 9 * g.tp;
    Cx<double>* pre = A.prefix[p] + (size_t)l * 9 * g.tp;
    P = ident<double>();
    for (int t = 0; t < g.T; ++t) {
      const int sl = slot_of(g, t);
#pragma unroll
      for (int k = 0; k < 9; ++k) pre[k * g.tp + sl] = P.e[k];
      P = matmul(P, ldmat(u, g.tp, sl));
    }
  }
  Mat3<double> B, Bi;
#pragma unroll
  for (int k = 0; k < 9; ++k)
    B.e[k] = mk<double>((k % 4 == 0 ? 1.0 : 0.0) - A.c * P.e[k].re, -A.c * P.e[k].im);
  const Cx<double> det = inverse3(B, Bi);
  A.ld[i] = 0.5 * log(det.re * det.re + det.im * det.im);
  const Mat3<double> Z = matmul(P, Bi);
#pragma unroll
  for (int k = 0; k < 9; ++k) A.z0[(size_t)i * 9 + k] = mk<double>(A.mu_pow * Z.e[k].re, A.mu_pow * Z.e[k].im);
}

// F^a = coef Re Tr[i T_a Z] = -coef Im Tr[T_a Z] for the halved Gell-Mann matrices T_a
__device__ __forceinline__ void project8(const Mat3<double>& Z, double coef, double* out) {
  const Cx<double>* z = Z.e;
  const double tr[8] = {
      0.5 * (z[1].im + z[3].im),
      0.5 * (z[1].re - z[3].re),
      0.5 * (z[0].im - z[4].im),
      0.5 * (z[2].im + z[6].im),
      0.5 * (z[2].re - z[6].re),
      0.5 * (z[5].im + z[7].im),
      0.5 * (z[5].re - z[7].re),
      (z[0].im + z[4].im - 2.0 * z[8].im) / (2.0 * sqrt(3.0)),
  };
#pragma unroll
  for (int a = 0; a < 8; ++a) out[a] = -coef * tr[a];
}

__global__ void __launch_bounds__(kSiteBlock) k_tdet_force(const DetArgs A) {
  const Geom& g = A.g;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)2 * g.Nl * g.tp) return;
  const int sl = (int)(i % g.tp);
  const int l = (int)((i / g.tp) % g.Nl);
  const int p = (int)(i / ((size_t)g.tp * g.Nl));
  const int t = (sl % g.lpl) * g.n + sl / g.lpl;  // inverse of slot_of
  if (t >= g.T) return;                            // padding slot
  const Cx<double>* rot = A.axial ? A.ut[p] : A.prefix[p];
  const Mat3<double> G = ldmat(rot + (size_t)l * 9 * g.tp, g.tp, sl);
  const Mat3<double> Z0 = ldmat(A.z0 + ((size_t)p * g.Nl + l) * 9, 1, 0);
  const Mat3<double> Z = matmul(dagger(G), matmul(Z0, G));
  int x, y, z;
  line_coords(g, p, l, x, y, z);
  const size_t site = (size_t)x + g.L * ((size_t)y + g.L * ((size_t)z + (size_t)g.L * t));
  double* f = A.F + site * 32;
#pragma unroll
  for (int k = 0; k < 24; ++k) f[k] = 0.0;
  project8(Z, A.coef, f + 24);
}

// out = 4 (sum_i ld[i] + n 3 N_t log mu), summed in a fixed order
__global__ void __launch_bounds__(kSumBlock) k_tdet_sum(const double* __restrict__ ld, int n, double log_mu_term,
                                                       double* out) {
  __shared__ double s[kSumBlock];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kSumBlock) acc += ld[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kSumBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = 4.0 * (s[0] + log_mu_term);
}

bool on_device(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int temporal_logdet(wf_handle* h, double* logdet, double* F) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  const Geom& g = h->g;
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  cudaStream_t s = h->stream;
  DetArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = g;
  a.axial = h->axial ? 1 : 0;
  a.c = g.bc * std::pow(g.mu, -(double)g.T);
  a.mu_pow = std::pow(g.mu, -(double)g.T);
  a.coef = -4.0 * g.bc;
  Cx<double>* prefix = a.axial ? nullptr : h->buf<Cx<double>>("det_prefix", (size_t)2 * g.Nl * 9 * g.tp);
  for (int p = 0; p < 2; ++p) {
    a.ut[p] = h->ut64[p].as<Cx<double>>();
    a.pl[p] = h->pl64[p].as<Cx<double>>();
    a.prefix[p] = prefix ? prefix + (size_t)p * g.Nl * 9 * g.tp : nullptr;
  }
  a.ld = h->buf<double>("det_ld", (size_t)2 * g.Nl + 1);
  a.z0 = h->buf<Cx<double>>("det_z0", (size_t)2 * g.Nl * 9);
  {
    Prof P(h, "tdet_line_f64");
    k_tdet_line<<<(2 * g.Nl + kLineBlock - 1) / kLineBlock, kLineBlock, 0, s>>>(a);
    WF_CUDA(cudaGetLastError());
  }
  if (logdet) {
    double* out = a.ld + 2 * g.Nl;
    {
      Prof P(h, "tdet_sum_f64");
      k_tdet_sum<<<1, kSumBlock, 0, s>>>(a.ld, 2 * g.Nl, 2.0 * g.Nl * 3.0 * g.T * std::log(g.mu), out);
      WF_CUDA(cudaGetLastError());
    }
    WF_CUDA(cudaMemcpyAsync(logdet, out, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  if (F) {
    const bool staged = !on_device(F);
    a.F = staged ? h->buf<double>("stage_force", V * 32) : F;
    const size_t n = (size_t)2 * g.Nl * g.tp;
    {
      Prof P(h, "tdet_force_f64");
      k_tdet_force<<<(unsigned)((n + kSiteBlock - 1) / kSiteBlock), kSiteBlock, 0, s>>>(a);
      WF_CUDA(cudaGetLastError());
    }
    if (staged) WF_CUDA(cudaMemcpyAsync(F, a.F, V * 32 * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  WF_CUDA(cudaStreamSynchronize(s));
  return WF_OK;
}

}  // namespace

extern "C" int wf_temporal_logdet(wf_handle_t* h, double* logdet, double* F) {
  if (!h) return WF_EINVAL;
  h->err.clear();
  try {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) WF_CUDA(cudaSetDevice(h->device));
    return temporal_logdet(h, logdet, F);
  } catch (const Error& e) {
    h->err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    h->err = e.what();
    return WF_ECUDA;
  } catch (...) {
    h->err = "unknown error";
    return WF_ECUDA;
  }
}
