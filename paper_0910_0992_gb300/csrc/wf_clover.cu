// The clover (SW) term of §II and its application, for the partially preconditioned clover
// operator with 3-D ILU (§II.B, Eq. TPrecPartial; App. B):
//
//   A(x) = -[ (c_t / 2) sum_i sigma_i0 F_i0(x) + (c_s / 2) sum_{i<j} sigma_ij F_ij(x) ],
//   sigma_mu nu = [gamma_mu, gamma_nu] / 2,   F_mu nu = (Q_mu nu - Q_mu nu^dag) / 8 less its trace,
//
// Q_mu nu(x) the sum of the four plaquette leaves of the mu nu plane that start and end at x,
// all with the orientation of U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag; one term per plane.
// A is hermitian and commutes with gamma_5 = -[[0, 1], [1, 0]] (spin halves u = spins 0-1,
// l = spins 2-3 of the Dirac-Pauli basis), so in the chiral basis a = (u + l)/sqrt 2,
// b = (u - l)/sqrt 2 it is two 6x6 blocks A_a, A_b. They are stored per 3-D parity as
// H_k = A_k / 2 in [Nl][2][36][tp] (slot-contiguous, like the links) and applied as
//   (A psi)_u = H_a (u + l) + H_b (u - l),   (A psi)_l = H_a (u + l) - H_b (u - l),
// two 6x6 complex products per site (App. B counts C(A) = 522 FLOPs for this block form).
//
// Build (FP64, once per gauge field): k_clover_field, one thread per site and plane, forms F from
// the lexicographic links and rotates it into the axial frame when the handle works there
// (F -> g F g^dag, g the frame rotation of the site); k_clover_blocks, one thread per entry of
// H_a, H_b, sums the six planes' F against the chiral blocks of sigma (the host folds the
// coefficients -c/2 and the 1/2 of H into those 2x2 blocks). For the 4-D Schur comparator,
// k_clover_eo4 stores the blocks of mu + A and of (mu + A)^-1 in the 4-D even-odd layout.
#include <cmath>
#include <complex>
#include <cstring>

#include "../../include/wf.h"
#include "wf_internal.h"
#include "wf_line.cuh"

namespace wf {

namespace {

constexpr int kBlock = 256;

// the six planes: (x, y), (x, z), (y, z) spatial, then (x, t), (y, t), (z, t)
__constant__ int c_plane_mu[6] = {0, 0, 1, 0, 1, 2};
__constant__ int c_plane_nu[6] = {1, 2, 2, 3, 3, 3};

struct CloverW {
  double re[6][2][2][2];  // [plane][chiral block][s][s']: coefficient x chiral block of sigma x 1/2
  double im[6][2][2][2];
};

__device__ __forceinline__ void site_xyzt(const Geom& g, size_t site, int& x, int& y, int& z, int& t) {
  x = (int)(site % g.L);
  y = (int)((site / g.L) % g.L);
  z = (int)((site / ((size_t)g.L * g.L)) % g.L);
  t = (int)(site / ((size_t)g.L * g.L * g.L));
}

__device__ __forceinline__ size_t site_of(const Geom& g, int x, int y, int z, int t) {
  return (size_t)x + g.L * ((size_t)y + g.L * ((size_t)z + (size_t)g.L * t));
}

// U_dir at the site c + (step_a along a) + (step_b along b), periodic
__device__ Mat3<double> link_at(const Geom& g, const Cx<double>* __restrict__ U, const int c[4], int dir, int a,
                                int sa, int b, int sb) {
  int q[4] = {c[0], c[1], c[2], c[3]};
  const int ext[4] = {g.L, g.L, g.L, g.T};
  q[a] = (q[a] + sa + ext[a]) % ext[a];
  q[b] = (q[b] + sb + ext[b]) % ext[b];
  const Cx<double>* p = U + (site_of(g, q[0], q[1], q[2], q[3]) * 4 + dir) * 9;
  Mat3<double> M;
#pragma unroll
  for (int k = 0; k < 9; ++k) M.e[k] = p[k];
  return M;
}

__global__ void __launch_bounds__(kBlock) k_clover_field(const Geom g, const Cx<double>* __restrict__ U,
                                                         const Cx<double>* __restrict__ rot0,
                                                         const Cx<double>* __restrict__ rot1, Cx<double>* F) {
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= V * 6) return;
  const int plane = (int)(i % 6);
  const size_t site = i / 6;
  int c[4];
  site_xyzt(g, site, c[0], c[1], c[2], c[3]);
  const int mu = c_plane_mu[plane], nu = c_plane_nu[plane];
  // the four leaves at x, one orientation
  Mat3<double> Q = matmul(matmul(link_at(g, U, c, mu, mu, 0, nu, 0), link_at(g, U, c, nu, mu, 1, nu, 0)),
                          matmul(dagger(link_at(g, U, c, mu, mu, 0, nu, 1)), dagger(link_at(g, U, c, nu, mu, 0, nu, 0))));
  Mat3<double> q2 = matmul(matmul(link_at(g, U, c, nu, mu, 0, nu, 0), dagger(link_at(g, U, c, mu, mu, -1, nu, 1))),
                           matmul(dagger(link_at(g, U, c, nu, mu, -1, nu, 0)), link_at(g, U, c, mu, mu, -1, nu, 0)));
  Mat3<double> q3 = matmul(matmul(dagger(link_at(g, U, c, mu, mu, -1, nu, 0)), dagger(link_at(g, U, c, nu, mu, -1, nu, -1))),
                           matmul(link_at(g, U, c, mu, mu, -1, nu, -1), link_at(g, U, c, nu, mu, 0, nu, -1)));
  Mat3<double> q4 = matmul(matmul(dagger(link_at(g, U, c, nu, mu, 0, nu, -1)), link_at(g, U, c, mu, mu, 0, nu, -1)),
                           matmul(link_at(g, U, c, nu, mu, 1, nu, -1), dagger(link_at(g, U, c, mu, mu, 0, nu, 0))));
#pragma unroll
  for (int k = 0; k < 9; ++k) Q.e[k] = Q.e[k] + q2.e[k] + q3.e[k] + q4.e[k];
  // F = (Q - Q^dag) / 8, trace removed
  Mat3<double> Fm;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const Cx<double> a = Q.e[3 * r + s], b = Q.e[3 * s + r];
      Fm.e[3 * r + s] = mk<double>(0.125 * (a.re - b.re), 0.125 * (a.im + b.im));
    }
  const double tr_im = (Fm.e[0].im + Fm.e[4].im + Fm.e[8].im) / 3.0;  // the trace is imaginary
#pragma unroll
  for (int k = 0; k < 9; k += 4) Fm.e[k].im -= tr_im;
  if (rot0) {
    const int p = (c[0] + c[1] + c[2]) & 1;
    const Cx<double>* rot = p ? rot1 : rot0;
    const Mat3<double> G = ldmat(rot + (size_t)line_of(g, c[0], c[1], c[2]) * 9 * g.tp, g.tp, slot_of(g, c[3]));
    Fm = matmul(G, matmul(Fm, dagger(G)));
  }
  Cx<double>* out = F + i * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) out[k] = Fm.e[k];
}

__global__ void __launch_bounds__(kBlock) k_clover_blocks(const Geom g, const CloverW W, const Cx<double>* __restrict__ F,
                                                          Cx<double>* H0, Cx<double>* H1) {
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= V * 72) return;
  const int e = (int)(i % 36);
  const int k = (int)((i / 36) % 2);
  const size_t site = i / 72;
  const int row = e / 6, col = e % 6;
  const int s = row / 3, cr = row % 3, s2 = col / 3, cc = col % 3;
  Cx<double> acc = czero<double>();
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const Cx<double> w = mk<double>(W.re[p][k][s][s2], W.im[p][k][s][s2]);
    acc = cfma(acc, w, F[(site * 6 + p) * 9 + 3 * cr + cc]);
  }
  int x, y, z, t;
  site_xyzt(g, site, x, y, z, t);
  Cx<double>* H = ((x + y + z) & 1) ? H1 : H0;
  H[(((size_t)line_of(g, x, y, z) * 2 + k) * 36 + e) * g.tp + slot_of(g, t)] = acc;
}

// out = acc + alpha H-blocks in (acc may be null: out = alpha H in) on one parity, all right-hand
// sides. Line layout (EO = false): fields [rhs][Nl][12][tp], blocks [Nl][2][36][tp], padding slots
// (t >= T) kept at the accumulator or zero. 4-D even-odd layout (EO = true): fields
// [rhs][L^3][12][T/2], blocks [L^3][2][36][T/2], no padding.
template <typename R, bool EO>
__global__ void __launch_bounds__(kBlock) k_clover_apply(const Geom g, const Cx<R>* __restrict__ H,
                                                         const Cx<R>* __restrict__ in, Cx<R>* out,
                                                         const Cx<R>* acc, R alpha, int nrhs) {
  const int outer = EO ? g.L * g.L * g.L : g.Nl;
  const int inner = EO ? g.T / 2 : g.tp;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nrhs * outer * inner) return;
  const int sl = (int)(i % inner);
  const int l = (int)((i / inner) % outer);
  const size_t base = (i / inner) * NSPIN_C * inner + sl;  // ((rhs outer + l) 12) inner + slot
  if (!EO) {
    const int t = (sl % g.lpl) * g.n + sl / g.lpl;
    if (t >= g.T) {  // padding slot: keep it at the accumulator (zero without one)
#pragma unroll
      for (int c = 0; c < NSPIN_C; ++c) out[base + (size_t)c * inner] = acc ? acc[base + (size_t)c * inner] : czero<R>();
      return;
    }
  }
  Cx<R> sv[6], dv[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const Cx<R> u = in[base + (size_t)c * inner], lo = in[base + (size_t)(c + 6) * inner];
    sv[c] = u + lo;
    dv[c] = u - lo;
  }
  const Cx<R>* Ha = H + ((size_t)l * 2) * 36 * inner + sl;
  const Cx<R>* Hb = Ha + (size_t)36 * inner;
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    Cx<R> ya = czero<R>(), yb = czero<R>();
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      ya = cfma(ya, Ha[(size_t)(6 * r + c) * inner], sv[c]);
      yb = cfma(yb, Hb[(size_t)(6 * r + c) * inner], dv[c]);
    }
    Cx<R> up = alpha * (ya + yb), lo = alpha * (ya - yb);
    if (acc) {
      up = up + acc[base + (size_t)r * inner];
      lo = lo + acc[base + (size_t)(r + 6) * inner];
    }
    out[base + (size_t)r * inner] = up;
    out[base + (size_t)(r + 6) * inner] = lo;
  }
}

// The 4-D even-odd blocks of mu + A and of its inverse, from the line-layout blocks H = A_k / 2:
// one thread per site and chiral block; B = mu 1 + A_k (6x6), B^-1 by Gauss-Jordan elimination
// with partial pivoting; stored halved like H. Sets *singular when a pivot vanishes.
__global__ void __launch_bounds__(128) k_clover_eo4(const Geom g, double mu, const Cx<double>* __restrict__ H0,
                                                    const Cx<double>* __restrict__ H1, Cx<double>* M0, Cx<double>* M1,
                                                    Cx<double>* Mi0, Cx<double>* Mi1, int* singular) {
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= V * 2) return;
  const int k = (int)(i % 2);
  const size_t site = i / 2;
  int x, y, z, t;
  site_xyzt(g, site, x, y, z, t);
  const Cx<double>* H = (((x + y + z) & 1) ? H1 : H0) + (((size_t)line_of(g, x, y, z) * 2 + k) * 36) * g.tp +
                        slot_of(g, t);
  const int Th = g.T / 2;
  const size_t s3 = (size_t)x + g.L * ((size_t)y + g.L * z);
  const size_t ob = ((s3 * 2 + k) * 36) * Th + t / 2;
  const bool odd4 = ((x + y + z + t) & 1) != 0;
  Cx<double>* M = odd4 ? M1 : M0;
  Cx<double>* Mi = odd4 ? Mi1 : Mi0;
  Cx<double> a[6][12];  // [B | 1]
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 6; ++c) {
      const Cx<double> h = H[(size_t)(6 * r + c) * g.tp];
      a[r][c] = mk<double>(2.0 * h.re + (r == c ? mu : 0.0), 2.0 * h.im);
      a[r][c + 6] = mk<double>(r == c ? 1.0 : 0.0, 0.0);
      M[(size_t)(6 * r + c) * Th + ob] = mk<double>(0.5 * a[r][c].re, 0.5 * a[r][c].im);
    }
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    double best = a[c][c].re * a[c][c].re + a[c][c].im * a[c][c].im;
    for (int r = c + 1; r < 6; ++r) {
      const double m = a[r][c].re * a[r][c].re + a[r][c].im * a[r][c].im;
      if (m > best) {
        best = m;
        piv = r;
      }
    }
    if (!(best > 1e-24)) {
      atomicExch(singular, 1);
      return;
    }
    if (piv != c)
      for (int j = 0; j < 12; ++j) {
        const Cx<double> tmp = a[c][j];
        a[c][j] = a[piv][j];
        a[piv][j] = tmp;
      }
    const Cx<double> inv = mk<double>(a[c][c].re / best, -a[c][c].im / best);
    for (int j = 0; j < 12; ++j) a[c][j] = cmul(a[c][j], inv);
    for (int r = 0; r < 6; ++r) {
      if (r == c) continue;
      const Cx<double> f = a[r][c];
      for (int j = 0; j < 12; ++j) a[r][j] = a[r][j] - cmul(f, a[c][j]);
    }
  }
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 6; ++c) Mi[(size_t)(6 * r + c) * Th + ob] = mk<double>(0.5 * a[r][c + 6].re, 0.5 * a[r][c + 6].im);
}

// out = in with the spin halves exchanged (the Dirac-Pauli gamma_5 up to its sign)
template <typename R>
__global__ void __launch_bounds__(kBlock) k_swap_halves(const Cx<R>* __restrict__ in, Cx<R>* __restrict__ out, size_t n,
                                                        int tp) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)((i / tp) % NSPIN_C);
  out[i] = in[c < 6 ? i + (size_t)6 * tp : i - (size_t)6 * tp];
}

unsigned grid_of(size_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// Dirac-Pauli gamma matrices: gamma_k = [[0, -i s_k], [i s_k, 0]], gamma_t = diag(1, 1, -1, -1)
using cd = std::complex<double>;
void gamma_dp(int mu, cd G[4][4]) {
  const cd I(0, 1);
  const cd s[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) G[r][c] = 0;
  if (mu == 3) {
    G[0][0] = G[1][1] = 1;
    G[2][2] = G[3][3] = -1;
    return;
  }
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      G[r][c + 2] = -I * s[mu][r][c];
      G[r + 2][c] = I * s[mu][r][c];
    }
}

CloverW clover_weights(double c_s, double c_t) {
  static const int pmu[6] = {0, 0, 1, 0, 1, 2}, pnu[6] = {1, 2, 2, 3, 3, 3};
  CloverW W;
  std::memset(&W, 0, sizeof(W));
  for (int p = 0; p < 6; ++p) {
    cd A[4][4], B[4][4], S[4][4];
    gamma_dp(pmu[p], A);
    gamma_dp(pnu[p], B);
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        cd ab = 0, ba = 0;
        for (int k = 0; k < 4; ++k) {
          ab += A[r][k] * B[k][c];
          ba += B[r][k] * A[k][c];
        }
        S[r][c] = 0.5 * (ab - ba);
      }
    const double coef = -0.5 * (p < 3 ? c_s : c_t);
    for (int s = 0; s < 2; ++s)
      for (int s2 = 0; s2 < 2; ++s2) {
        const cd uu = S[s][s2], ul = S[s][s2 + 2], lu = S[s + 2][s2], ll = S[s + 2][s2 + 2];
        const cd blk[2] = {0.5 * (uu + ul + lu + ll), 0.5 * (uu - ul - lu + ll)};
        const cd off = 0.5 * (uu - ul + lu - ll);  // vanishes: sigma commutes with gamma_5
        if (std::abs(off) > 1e-12) throw Error(WF_EINVAL, "clover: sigma does not commute with gamma_5");
        for (int k = 0; k < 2; ++k) {
          const cd w = 0.5 * coef * blk[k];
          W.re[p][k][s][s2] = w.real();
          W.im[p][k][s][s2] = w.imag();
        }
      }
  }
  return W;
}

}  // namespace

void launch_clover_build(const Geom& g, const Cx<double>* U_lex, const Cx<double>* rot[2], double c_s, double c_t,
                         Cx<double>* F_scratch, Cx<double>* H[2], cudaStream_t s) {
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const CloverW W = clover_weights(c_s, c_t);
  k_clover_field<<<grid_of(V * 6), kBlock, 0, s>>>(g, U_lex, rot ? rot[0] : nullptr, rot ? rot[1] : nullptr, F_scratch);
  WF_CUDA(cudaGetLastError());
  k_clover_blocks<<<grid_of(V * 72), kBlock, 0, s>>>(g, W, F_scratch, H[0], H[1]);
  WF_CUDA(cudaGetLastError());
}

template <typename R>
void launch_clover_apply(const Geom& g, const Cx<R>* H, const Cx<R>* in, Cx<R>* out, const Cx<R>* acc, double alpha,
                         int nrhs, cudaStream_t s) {
  k_clover_apply<R, false><<<grid_of((size_t)nrhs * g.Nl * g.tp), kBlock, 0, s>>>(g, H, in, out, acc, (R)alpha, nrhs);
  WF_CUDA(cudaGetLastError());
}
template void launch_clover_apply<float>(const Geom&, const Cx<float>*, const Cx<float>*, Cx<float>*,
                                         const Cx<float>*, double, int, cudaStream_t);
template void launch_clover_apply<double>(const Geom&, const Cx<double>*, const Cx<double>*, Cx<double>*,
                                          const Cx<double>*, double, int, cudaStream_t);

template <typename R>
void launch_clover_apply_eo(const Geom& g, const Cx<R>* H, const Cx<R>* in, Cx<R>* out, const Cx<R>* acc,
                            double alpha, int nrhs, cudaStream_t s) {
  const size_t n = (size_t)nrhs * g.L * g.L * g.L * (g.T / 2);
  k_clover_apply<R, true><<<grid_of(n), kBlock, 0, s>>>(g, H, in, out, acc, (R)alpha, nrhs);
  WF_CUDA(cudaGetLastError());
}
template void launch_clover_apply_eo<float>(const Geom&, const Cx<float>*, const Cx<float>*, Cx<float>*,
                                            const Cx<float>*, double, int, cudaStream_t);
template void launch_clover_apply_eo<double>(const Geom&, const Cx<double>*, const Cx<double>*, Cx<double>*,
                                             const Cx<double>*, double, int, cudaStream_t);

void launch_clover_eo4_build(const Geom& g, const Cx<double>* H[2], Cx<double>* M[2], Cx<double>* Minv[2],
                             int* singular, cudaStream_t s) {
  const size_t n = (size_t)g.L * g.L * g.L * g.T * 2;
  k_clover_eo4<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, g.mu, H[0], H[1], M[0], M[1], Minv[0], Minv[1], singular);
  WF_CUDA(cudaGetLastError());
}

template <typename R>
void launch_swap_halves(const Cx<R>* in, Cx<R>* out, size_t n, int tp, cudaStream_t s) {
  k_swap_halves<R><<<grid_of(n), kBlock, 0, s>>>(in, out, n, tp);
  WF_CUDA(cudaGetLastError());
}
template void launch_swap_halves<float>(const Cx<float>*, Cx<float>*, size_t, int, cudaStream_t);
template void launch_swap_halves<double>(const Cx<double>*, Cx<double>*, size_t, int, cudaStream_t);

}  // namespace wf
