// Pseudofermion force of the temporally preconditioned operator: the link outer products.
//
// S = phi^dag (M-hat^dag M-hat)^-1 phi, X = (M-hat^dag M-hat)^-1 phi, Y = M-hat X and
// dS = -2 Re(Y^dag dM-hat X) with M-hat = 1 - gamma_f^-2 C_L^o D^oe C_R^e C_L^e D^eo C_R^o
// (§II.B, Eq. TPrecFull; the paper defers the HMC force to later work, §IV). The host
// builds the right chain v_k and the left chain w_k (applications of C_L, C_R, D_s and their
// adjoints); these kernels turn pairs of chain vectors into, per link, the 3x3 matrix Z with
// dS/d eps_a = 2 gamma_f^-2 Re Tr[i T_a Z] for U -> exp(i eps T_a) U, T_a = lambda_a / 2:
//   temporal link U_t(t) of a line, from a C_L factor (pair a, b: P_- halves) and a C_R factor
//   (pair c, e: P_+ halves):
//     Z = s(t) sum_{P_- spins} (U_t(t) b(t+1)) a(t)^dag - s(t) sum_{P_+ spins} e(t) (U_t(t) c(t+1))^dag
//   spatial link U_k(x), from the two D_s factors:
//     Z = sum_spins (U_k v(x+k)) (P^-_k w(x))^dag - v'(x) (U_k P^+_k w'(x+k))^dag
// In the axial frame the kernels work with the rotated links and return Z to the caller's
// gauge with the rotation of the link's base site: Z <- g(x)^dag Z g(x).
#include "wf_internal.h"
#include "wf_line.cuh"

namespace wf {


__device__ __forceinline__ Vec3<double> fvec(const Cx<double>* f, size_t line_base, int comp0, int tp, int sl) {
  return ldvec(f + line_base + (size_t)comp0 * tp, tp, sl);
}

// acc += x y^dag
__device__ __forceinline__ void outer_acc(Mat3<double>& Z, const Vec3<double>& x, const Vec3<double>& y, double s) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<double> p = cfmaconj(czero<double>(), y.c[j], x.c[i]);  // x_i conj(y_j)
      Z.e[3 * i + j] = Z.e[3 * i + j] + s * p;
    }
}

// F^a = coef Re Tr[i T_a Z] = -coef Im Tr[T_a Z], T_a = lambda_a / 2 (Gell-Mann)
__device__ __forceinline__ void project(const Mat3<double>& Z, double coef, double* out) {
  const Cx<double>* z = Z.e;
  auto im = [](Cx<double> v) { return v.im; };
  auto re = [](Cx<double> v) { return v.re; };
  // Tr[T_a Z] for the eight generators; only the imaginary part of i * (.) is needed
  const double t1 = im(z[3] + z[1]) * 0.5;
  const double t2 = (re(z[1]) - re(z[3])) * 0.5;   // Im((-i z10 + i z01)/2)
  const double t3 = im(z[0] - z[4]) * 0.5;
  const double t4 = im(z[6] + z[2]) * 0.5;
  const double t5 = (re(z[2]) - re(z[6])) * 0.5;
  const double t6 = im(z[7] + z[5]) * 0.5;
  const double t7 = (re(z[5]) - re(z[7])) * 0.5;
  const double t8 = (im(z[0]) + im(z[4]) - 2.0 * im(z[8])) / (2.0 * sqrt(3.0));
  out[0] = -coef * t1;
  out[1] = -coef * t2;
  out[2] = -coef * t3;
  out[3] = -coef * t4;
  out[4] = -coef * t5;
  out[5] = -coef * t6;
  out[6] = -coef * t7;
  out[7] = -coef * t8;
}

__device__ __forceinline__ Mat3<double> to_caller_gauge(const Mat3<double>& Z, const ForceArgs& A, int l, int sl) {
  if (!A.axial) return Z;
  const Mat3<double> G = ldmat(A.ut + (size_t)l * 9 * A.g.tp, A.g.tp, sl);
  return matmul(dagger(G), matmul(Z, G));
}

__device__ __forceinline__ size_t lex_site(const Geom& g, int x, int y, int z, int t) {
  return (size_t)x + g.L * ((size_t)y + g.L * ((size_t)z + (size_t)g.L * t));
}

__global__ void k_force_temporal(const ForceArgs A) {
  const Geom& g = A.g;
  const size_t total = (size_t)g.Nl * g.T;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int t = (int)(i % g.T);
  const int l = (int)(i / g.T);
  const int tp = g.tp;
  const int sl = slot_of(g, t);
  const int tn = t == g.T - 1 ? 0 : t + 1;
  const int sln = slot_of(g, tn);
  const double sg = t == g.T - 1 ? A.bc : 1.0;
  const size_t lb = (size_t)l * NSPIN_C * tp;
  Mat3<double> U;
  bool unit = false;
  if (A.axial) {
    if (t == g.T - 1)
      U = ldmat(A.pl + (size_t)l * 9, 1, 0);
    else
      unit = true;
  } else {
    U = ldmat(A.ut + (size_t)l * 9 * tp, tp, sl);
  }
  Mat3<double> Z;
#pragma unroll
  for (int k = 0; k < 9; ++k) Z.e[k] = czero<double>();
  // C_L factor: spins 2, 3 (P_-)
#pragma unroll
  for (int s = 2; s < 4; ++s) {
    Vec3<double> bn = fvec(A.b, lb, 3 * s, tp, sln);
    Vec3<double> ub = unit ? bn : matvec(U, bn);
    outer_acc(Z, ub, fvec(A.a, lb, 3 * s, tp, sl), sg);
  }
  // C_R factor: spins 0, 1 (P_+)
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    Vec3<double> cn = fvec(A.c, lb, 3 * s, tp, sln);
    Vec3<double> uc = unit ? cn : matvec(U, cn);
    outer_acc(Z, fvec(A.e, lb, 3 * s, tp, sl), uc, -sg);
  }
  Z = to_caller_gauge(Z, A, l, sl);
  int x, y, z;
  line_coords(g, A.parity, l, x, y, z);
  project(Z, A.coef, A.F + (lex_site(g, x, y, z, t) * 4 + 3) * 8);
}

__global__ void k_force_spatial(const ForceArgs A) {
  const Geom& g = A.g;
  const size_t total = (size_t)g.Nl * g.T;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int t = (int)(i % g.T);
  const int l = (int)(i / g.T);
  const int tp = g.tp;
  const int sl = slot_of(g, t);
  int nb[6];
  neighbour_lines(g, A.parity, l, nb);
  int x, y, z;
  line_coords(g, A.parity, l, x, y, z);
  const size_t lb = (size_t)l * NSPIN_C * tp;
  for (int k = 0; k < 3; ++k) {
    const size_t nbb = (size_t)nb[2 * k] * NSPIN_C * tp;
    const Mat3<double> U = ldmat(A.us_p + ((size_t)k * g.Nl + l) * NLINK_C * tp, tp, sl);
    // spinors: w(x), v(x+k), vr(x), wr(x+k)
    Vec3<double> w[4], v[4], vr[4], wr[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      w[s] = fvec(A.w, lb, 3 * s, tp, sl);
      v[s] = fvec(A.v, nbb, 3 * s, tp, sl);
      vr[s] = fvec(A.vr, lb, 3 * s, tp, sl);
      wr[s] = fvec(A.wr, nbb, 3 * s, tp, sl);
    }
    // P^-_k w = ((h), -i sigma_k h) / 2 with h = w_up + i sigma_k w_lo; P^+_k wr = ((h'), i sigma_k h') / 2
    Vec3<double> s0, s1, h0, h1, r0, r1;
    isigma(k, w[2], w[3], s0, s1);
    h0 = vscale(0.5, vadd(w[0], s0));
    h1 = vscale(0.5, vadd(w[1], s1));
    isigma(k, h0, h1, r0, r1);
    Vec3<double> pm[4] = {h0, h1, vscale(-1.0, r0), vscale(-1.0, r1)};
    isigma(k, wr[2], wr[3], s0, s1);
    h0 = vscale(0.5, vaxpy(-1.0, s0, wr[0]));
    h1 = vscale(0.5, vaxpy(-1.0, s1, wr[1]));
    isigma(k, h0, h1, r0, r1);
    Vec3<double> pp[4] = {h0, h1, r0, r1};
    Mat3<double> Z;
#pragma unroll
    for (int e = 0; e < 9; ++e) Z.e[e] = czero<double>();
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      outer_acc(Z, matvec(U, v[s]), pm[s], 1.0);
      outer_acc(Z, vr[s], matvec(U, pp[s]), -1.0);
    }
    Z = to_caller_gauge(Z, A, l, sl);
    project(Z, A.coef, A.F + (lex_site(g, x, y, z, t) * 4 + k) * 8);
  }
}

void launch_force(const ForceArgs& a, cudaStream_t s) {
  const size_t total = (size_t)a.g.Nl * a.g.T;
  const int blocks = (int)((total + 127) / 128);
  k_force_temporal<<<blocks, 128, 0, s>>>(a);
  k_force_spatial<<<blocks, 128, 0, s>>>(a);
  WF_CUDA(cudaGetLastError());
}

}  // namespace wf
