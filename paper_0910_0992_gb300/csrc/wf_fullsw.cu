// Full SW temporal preconditioning (§II.A, the paragraphs on SW fermions; appendix "Full
// Preconditioning with Clover"): the temporal block Q = A + mu - D_t of every spatial line, the
// clover term included, is inverted whole, and the 3-D Schur operator on odd sites becomes
//
//   M-hat_full = 1 - gamma_f^-2 (Q^oo)^-1 D_s^oe (Q^ee)^-1 D_s^eo,
//
// the form of Eq. TPrecFull with the one-sided split C_L = Q^-1, C_R = 1 (any split of Q leaves
// Q-bar = 1). Its adjoint follows from the gamma_5-hermiticity of Q and D_s:
//   M-hat_full^dag = 1 - gamma_f^-2 gamma_5 D_s^oe (Q^ee)^-1 D_s^eo (Q^oo)^-1 gamma_5,
// with gamma_5 = -S (S exchanges the spin halves of the Dirac-Pauli basis), so the two signs cancel.
//
// Q on one line is block tridiagonal in time with 12x12 blocks, closed by two wrap couplings. The
// appendix writes Q = T_0 + V W^dag, T_0 the open chain and V W^dag the wrap (rank 12: the P_+ half
// of slot 0 couples to slot N_t - 1, the P_- half of slot N_t - 1 to slot 0; V carries -s U_w^dag
// and -s U_w, U_w the link from N_t - 1 to 0, s the boundary sign; W^dag = (P_-, 0, .., 0, P_+)),
// and inverts it by one Woodbury step
//   Q^-1 = T_0^-1 - T_0^-1 V Lambda W^dag T_0^-1,   Lambda = (1 + W^dag T_0^-1 V)^-1.
// The paper solves T_0 by an inner CG. Here T_0 is factored once per gauge field by block LU
// (the block Thomas recursion), which its projector couplings make cheap: with W_t the link from
// t to t + 1 (1 in the axial frame),
//   Sigma_0 = mu + A(0),
//   Sigma_t = mu + A(t) - [P_+ (x) W_{t-1}^dag] Sigma_{t-1}^-1 [P_- (x) W_{t-1}]   (t >= 1),
// so Sigma_t differs from the diagonal block only in its (P_+ rows, P_- columns) corner. One
// solve T_0 y = b is a forward sweep
//   z_0 = b_0,   z_t = b_t + [P_+ (x) W_{t-1}^dag] Sigma_{t-1}^-1 z_{t-1}
// (only the P_+ half of Sigma_{t-1}^-1 z_{t-1} is needed) and a backward sweep
//   y_{N_t-1} = Sigma_{N_t-1}^-1 z_{N_t-1},   y_t = Sigma_t^-1 (z_t + [P_- (x) W_t] y_{t+1}),
// and with Z = T_0^-1 V (12 columns, formed once with the factors) Q^-1 b takes one solve:
// chi = T_0^-1 b, c = Lambda W^dag chi (W^dag chi: the P_+ half of chi_{N_t-1} and the P_- half of
// chi_0), Q^-1 b = chi - Z c.
//
// Kernels. k_qinv_setup (one CTA per line, in the precision of the applies that use it: FP64, or
// FP32 from the FP32 gauge and clover copies, since FP32 solves correct against the FP64 true
// residual of M_SW and never need FP64 factors): Sigma_t^-1 for every t by Gauss-Jordan elimination
// with partial pivoting in shared memory, then the twelve columns of T_0^-1 V by the sweeps (one
// 16-lane group per column, the forward sweep's z in a global scratch array), kept as Z, then
// Lambda.
// k_qinv_apply: one 16-lane group per (line, right-hand side), lane r < 12 holding component
// r (= 3 spin + colour) of the current 12-vector; a sweep step is a 12x12 (6x12 in the forward
// sweep) product whose vector the group exchanges through shared memory; the correction chi - Z c
// has no serial chain. Lane r only ever needs
// row r of a block, so it streams its rows (and b_t) into a per-group ring in shared memory with
// cp.async several steps ahead of their use: the sweeps' serial chains then wait on shared memory
// and arithmetic, not on DRAM. Blocks are stored row-major per time slice, [line][t][r][k], so that
// a lane copies its row as 16-byte pieces.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/wf.h"
#include "wf_handle.h"
#include "wf_line.cuh"

namespace wf {

namespace {

constexpr int kGrp = 16;                       // lanes per 12-vector group
constexpr int kSetupThreads = 12 * kGrp;       // one group per column of V
constexpr int kBlk = 144;                      // entries of a 12x12 block
constexpr size_t kScratchBytes = 256u << 20;   // bound of the setup's sweep scratch per launch

template <typename R>
__device__ __forceinline__ Cx<R> cconj(Cx<R> a) { return mk<R>(a.re, -a.im); }

// row r of the 12x12 block B (element (r, k) at B[12 r + k]) times the group's vector v
template <typename R>
__device__ __forceinline__ Cx<R> row_times(const Cx<R>* __restrict__ B, int r, const Cx<R>* v) {
  Cx<R> acc = czero<R>();
#pragma unroll
  for (int k = 0; k < 12; ++k) acc = cfma(acc, B[12 * r + k], v[k]);
  return acc;
}

// One solve T_0 y = b on one line by a 16-lane group, as the setup runs it for the columns of V
// (the apply kernel has its own sweeps, fed ahead through shared memory): lane r < 12 holds
// component r, lanes 12-15 only join the group's barriers (mask). S: the line's Sigma_t^-1 blocks [T][144]; ut: the line's
// U_t [9][tp] (general frame; unused in the axial frame, where W_t = 1). rhs(t): component r of
// b_t; zst / zld: store / load component r of the forward sweep's z_t; out(t, y): component r of
// y_t, produced for t = N_t - 1 down to 0. sh: the group's 16-element exchange vector.
template <typename R, bool AX, class RhsF, class ZSt, class ZLd, class OutF>
__device__ __forceinline__ void t0_solve(const Cx<R>* __restrict__ S, const Cx<R>* __restrict__ ut, const Geom& g,
                                         int r, unsigned mask, Cx<R>* sh, RhsF rhs, ZSt zst, ZLd zld, OutF out) {
  const int T = g.T;
  const bool act = r < 12;
  const int sr = r / 3, cr = r - 3 * (r / 3);  // spin and colour of component r
  Cx<R> z = act ? rhs(0) : czero<R>();
  if (act) zst(0, z);
  for (int t = 1; t < T; ++t) {
    if (act) sh[r] = z;
    __syncwarp(mask);
    const Cx<R> w = r < 6 ? row_times(S + (size_t)(t - 1) * kBlk, r, sh) : czero<R>();
    __syncwarp(mask);
    if (r < 6) sh[r] = w;
    __syncwarp(mask);
    z = act ? rhs(t) : czero<R>();
    if (r < 6) {
      if (AX) {
        z = z + sh[r];
      } else {  // + (W_{t-1}^dag w) on spin sr: sum_c conj(W[c][cr]) w[3 sr + c]
        const int sl = slot_of(g, t - 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) z = cfmaconj(z, ut[(size_t)(3 * c + cr) * g.tp + sl], sh[3 * sr + c]);
      }
    }
    __syncwarp(mask);
    if (act) zst(t, z);
  }
  if (act) sh[r] = z;
  __syncwarp(mask);
  Cx<R> y = act ? row_times(S + (size_t)(T - 1) * kBlk, r, sh) : czero<R>();
  if (act) out(T - 1, y);
  for (int t = T - 2; t >= 0; --t) {
    __syncwarp(mask);
    if (act) sh[r] = y;
    __syncwarp(mask);
    Cx<R> v = act ? zld(t) : czero<R>();
    if (act && r >= 6) {
      if (AX) {
        v = v + sh[r];
      } else {  // + (W_t y_{t+1}) on spin sr: sum_c W[cr][c] y[3 sr + c]
        const int sl = slot_of(g, t);
#pragma unroll
        for (int c = 0; c < 3; ++c) v = cfma(v, ut[(size_t)(3 * cr + c) * g.tp + sl], sh[3 * sr + c]);
      }
    }
    __syncwarp(mask);
    if (act) sh[r] = v;
    __syncwarp(mask);
    y = act ? row_times(S + (size_t)t * kBlk, r, sh) : czero<R>();
    if (act) out(t, y);
  }
  __syncwarp(mask);
}

// In-place inverse of the 12x12 left half of a[12][24] (right half: the identity on entry, the
// inverse on exit) by Gauss-Jordan elimination with partial pivoting; every thread of the CTA
// calls it. Returns false (the same on all threads) if a pivot is zero or not finite.
template <typename R>
__device__ bool gj_invert(Cx<R> (*a)[24], Cx<R>* fcol, int* piv, int tid, int nthreads) {
  const R lo = sizeof(R) == 8 ? R(1e-280) : R(1e-30), hi = sizeof(R) == 8 ? R(1e280) : R(1e30);
  for (int k = 0; k < 12; ++k) {
    if (tid == 0) {
      int p = k;
      R best = a[k][k].re * a[k][k].re + a[k][k].im * a[k][k].im;
      for (int i = k + 1; i < 12; ++i) {
        const R v = a[i][k].re * a[i][k].re + a[i][k].im * a[i][k].im;
        if (v > best) {
          best = v;
          p = i;
        }
      }
      piv[0] = p;
      piv[1] = (best > lo && best < hi) ? 0 : 1;  // also false for NaN
    }
    __syncthreads();
    if (piv[1]) return false;
    const int p = piv[0];
    if (p != k && tid < 24) {
      const Cx<R> tmp = a[k][tid];
      a[k][tid] = a[p][tid];
      a[p][tid] = tmp;
    }
    __syncthreads();
    const Cx<R> pv = a[k][k];
    __syncthreads();  // every thread has the pivot before row k changes
    const R d = R(1) / (pv.re * pv.re + pv.im * pv.im);
    const Cx<R> ip = mk<R>(pv.re * d, -pv.im * d);
    if (tid < 24) a[k][tid] = cmul(a[k][tid], ip);
    if (tid >= 32 && tid < 44) fcol[tid - 32] = a[tid - 32][k];  // rows != k: untouched above
    __syncthreads();
    for (int e = tid; e < 12 * 24; e += nthreads) {
      const int r = e / 24, c = e - 24 * (e / 24);
      if (r != k) a[r][c] = a[r][c] - cmul(fcol[r], a[k][c]);
    }
    __syncthreads();
  }
  return true;
}

template <typename R>
struct SetupArgs {
  Geom g;
  int line0;            // first line of this launch
  const Cx<R>* H;       // clover blocks of the parity [Nl][2][36][tp] (H_a, H_b = half the chiral
                        // blocks of A), or null: A = 0
  const Cx<R>* ut;      // general frame: U_t of the parity [Nl][9][tp]
  const Cx<R>* pl;      // axial frame: the boundary link P of every line [Nl][9]
  R s;                  // boundary sign
  Cx<R>* sinv;          // out: Sigma_t^-1 [Nl][T][144], row-major per block
  Cx<R>* lam;           // out: Lambda [Nl][144], row-major
  Cx<R>* zv;            // out: Z = T_0^-1 V [Nl][T][144], row-major per time slice
  Cx<R>* scratch;       // [lines of this launch][12][T][12]: forward sweeps of the columns of V
  int* singular;        // set to 1 if a block has no inverse
};

// The factorisation in precision R (FP64 for the FP64 applies and solves; FP32 ones use factors
// formed in FP32 from the FP32 gauge field and clover term)
template <typename R, bool AX>
__global__ void __launch_bounds__(kSetupThreads) k_qinv_setup(const SetupArgs<R> A) {
  __shared__ Cx<R> aug[12][24];
  __shared__ Cx<R> prev[kBlk];  // Sigma_{t-1}^-1, transposed
  __shared__ Cx<R> fcol[12];
  __shared__ Cx<R> wl[9];       // a link: W_{t-1} while factoring, then U_w
  __shared__ Cx<R> gsh[12][kGrp];
  __shared__ int piv[2];
  const Geom& g = A.g;
  const int tid = threadIdx.x;
  const int l = A.line0 + blockIdx.x;
  const int T = g.T, tp = g.tp;
  Cx<R>* S = A.sinv + (size_t)l * T * kBlk;
  const Cx<R>* ut = AX ? nullptr : A.ut + (size_t)l * 9 * tp;
  const Cx<R>* Hl = A.H ? A.H + (size_t)l * 72 * tp : nullptr;
  const R mu = (R)g.mu;

  // block LU of T_0
  for (int t = 0; t < T; ++t) {
    const int sl = slot_of(g, t);
    if (!AX && t > 0 && tid < 9) wl[tid] = ut[(size_t)tid * tp + slot_of(g, t - 1)];
    __syncthreads();
    if (tid < kBlk) {
      const int r = tid / 12, c = tid - 12 * (tid / 12);
      Cx<R> v = mk<R>(r == c ? mu : R(0), R(0));
      if (Hl) {  // A = [[H_a + H_b, H_a - H_b], [H_a - H_b, H_a + H_b]] on the (P_+, P_-) halves
        const int i = r % 6, j = c % 6;
        const Cx<R> ha = Hl[(size_t)(6 * i + j) * tp + sl], hb = Hl[(size_t)(36 + 6 * i + j) * tp + sl];
        v = (r < 6) == (c < 6) ? v + ha + hb : v + ha - hb;
      }
      if (t > 0 && r < 6 && c >= 6) {
        if (AX) {
          v = v - prev[12 * c + r];
        } else {  // sum_ab conj(W[a][cr]) Sigma^-1[(sr, a), (sc, b)] W[b][cc]
          const int sr = r / 3, cr = r % 3, sc = c / 3, cc = c % 3;
          Cx<R> acc = czero<R>();
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
              acc = acc + cmul(cmul(cconj(wl[3 * a + cr]), prev[12 * (3 * sc + b) + 3 * sr + a]), wl[3 * b + cc]);
          v = v - acc;
        }
      }
      aug[r][c] = v;
      aug[r][c + 12] = mk<R>(r == c ? R(1) : R(0), R(0));
    }
    __syncthreads();
    if (!gj_invert<R>(aug, fcol, piv, tid, kSetupThreads)) {
      if (tid == 0) atomicOr(A.singular, 1);
      return;
    }
    if (tid < kBlk) {
      const int r = tid / 12, k = tid - 12 * (tid / 12);
      const Cx<R> v = aug[r][k + 12];
      prev[12 * k + r] = v;
      S[(size_t)t * kBlk + 12 * r + k] = v;
    }
    __syncthreads();
  }

  // Z = T_0^-1 V and W^dag Z, one column j of V per group
  if (tid < 9) wl[tid] = AX ? A.pl[(size_t)l * 9 + tid] : ut[(size_t)tid * tp + slot_of(g, T - 1)];
  __syncthreads();
  const int j = tid / kGrp, r = tid % kGrp;
  const unsigned mask = 0xFFFFu << (tid & 16);
  Cx<R>* scr = A.scratch + ((size_t)blockIdx.x * 12 + j) * T * 12;
  const R ms = -A.s;
  auto rhs = [&](int t) -> Cx<R> {
    if (j < 6) {  // V_0 = -s P_+ (x) U_w^dag: rows of spin j / 3
      if (t == 0 && r < 6 && r / 3 == j / 3) return ms * cconj(wl[3 * (j % 3) + r % 3]);
    } else {      // V_{N_t-1} = -s P_- (x) U_w
      if (t == T - 1 && r >= 6 && r / 3 == j / 3) return ms * wl[3 * (r % 3) + j % 3];
    }
    return czero<R>();
  };
  auto zst = [&](int t, Cx<R> v) { scr[(size_t)t * 12 + r] = v; };
  auto zld = [&](int t) { return scr[(size_t)t * 12 + r]; };
  Cx<R> y0 = czero<R>(), yT = czero<R>();
  Cx<R>* Z = A.zv + (size_t)l * T * kBlk + 12 * r + j;
  auto column = [&](int t, Cx<R> v) {
    Z[(size_t)t * kBlk] = v;
    if (t == 0) y0 = v;
    if (t == T - 1) yT = v;
  };
  t0_solve<R, AX>(S, ut, g, r, mask, gsh[j], rhs, zst, zld, column);
  __syncthreads();
  if (r < 12) {  // 1 + W^dag T_0^-1 V, column j
    aug[r][j] = (r < 6 ? yT : y0) + mk<R>(r == j ? R(1) : R(0), R(0));
    aug[r][j + 12] = mk<R>(r == j ? R(1) : R(0), R(0));
  }
  __syncthreads();
  if (!gj_invert<R>(aug, fcol, piv, tid, kSetupThreads)) {
    if (tid == 0) atomicOr(A.singular, 1);
    return;
  }
  if (tid < kBlk) {
    const int rr = tid / 12, k = tid - 12 * (tid / 12);
    A.lam[(size_t)l * kBlk + 12 * rr + k] = aug[rr][k + 12];
  }
}

template <typename R>
struct QinvArgs {
  Geom g;
  int nrhs;
  const Cx<R>* in;     // [nrhs][Nl][12][tp], one 3-D parity
  Cx<R>* out;          // out = xpost + apost Q^-1 (S if swap_in) in; out != in
  const Cx<R>* xpost;  // null: out = Q^-1 in
  R apost;
  int swap_in;         // read in with the spin halves exchanged
  const Cx<R>* sinv;   // [Nl][T][144]
  const Cx<R>* lam;    // [Nl][144]
  const Cx<R>* zv;     // Z = T_0^-1 V [Nl][T][144]
  const Cx<R>* ut;     // general frame: U_t [Nl][9][tp]
  const Cx<R>* pl;     // axial frame: P [Nl][9]
  R s;                 // boundary sign
};

// per-lane asynchronous global -> shared copies (completion tracked per thread in commit groups)
template <typename R>
__device__ __forceinline__ void cp_async(Cx<R>* dst, const Cx<R>* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(__cvta_generic_to_global(src)), "n"((int)sizeof(Cx<R>))
               : "memory");
}
// 16 bytes: two FP32 or one FP64 complex element (both addresses 16-byte aligned), cached in L1
// so that the sources of one line on an SM share the rows
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}
// elements k and k + 1 of a 16-byte aligned row in shared memory
__device__ __forceinline__ void ld_pair(const Cx<float>* p, Cx<float>& a, Cx<float>& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = mk<float>(v.x, v.y);
  b = mk<float>(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const Cx<double>* p, Cx<double>& a, Cx<double>& b) {
  a = p[0];
  b = p[1];
}
// lane row of 12 block elements from global src (16-byte aligned) to shared dst
template <typename R>
__device__ __forceinline__ void cp_row(Cx<R>* dst, const Cx<R>* src) {
  constexpr int per = 16 / (int)sizeof(Cx<R>);
#pragma unroll
  for (int i = 0; i < 12; i += per) cp_async16(dst + i, src + i);
}
// row . v over 12 elements, two accumulators
template <typename R>
__device__ __forceinline__ Cx<R> row_dot(const Cx<R>* row, const Cx<R>* v) {
  Cx<R> a0 = czero<R>(), a1 = czero<R>();
#pragma unroll
  for (int k = 0; k < 12; k += 2) {
    Cx<R> m0, m1, v0, v1;
    ld_pair(row + k, m0, m1);
    ld_pair(v + k, v0, v1);
    a0 = cfma(a0, m0, v0);
    a1 = cfma(a1, m1, v1);
  }
  return a0 + a1;
}
// row . v with v in registers
template <typename R>
__device__ __forceinline__ Cx<R> row_dot_reg(const Cx<R>* row, const Cx<R> (&v)[12]) {
  Cx<R> a0 = czero<R>(), a1 = czero<R>();
#pragma unroll
  for (int k = 0; k < 12; k += 2) {
    Cx<R> m0, m1;
    ld_pair(row + k, m0, m1);
    a0 = cfma(a0, m0, v[k]);
    a1 = cfma(a1, m1, v[k + 1]);
  }
  return a0 + a1;
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kQGroups = 4;  // 16-lane groups per CTA of k_qinv_apply

// Ring of k_qinv_apply: depth (the steps whose operands are in flight; a shallower ring with more
// CTAs per SM measured slower) and elements per lane row (12 of a block, the step's other operand,
// and padding that keeps rows 16-byte aligned and 16-byte row reads free of bank conflicts)
template <typename R>
struct QRing {
  static constexpr int depth = sizeof(R) == 8 ? 4 : 6;
  static constexpr int row = sizeof(R) == 8 ? 13 : 14;
};
constexpr int kTMax = 256;  // longest time line

// Q^-1 per (line, right-hand side), one 16-lane group each: chi = T_0^-1 b by the two sweeps,
// then Q^-1 b = chi - Z c with c = Lambda W^dag chi, a pass with no serial chain. Every step takes
// lane r's row of a 12x12 block and one more operand (b_t, or the post-axpy operand) from a
// per-group ring of D steps in shared memory that the lane fills D - 1 steps ahead with cp.async;
// a lane reads only what it copied itself, so the ring needs no barrier. z_t and chi_t go through
// out and come back two steps ahead of their use.
template <typename R, bool AX>
__global__ void __launch_bounds__(kQGroups * kGrp) k_qinv_apply(const QinvArgs<R> A) {
  constexpr int D = QRing<R>::depth, RW = QRing<R>::row;
  __shared__ __align__(16) Cx<R> ring[kQGroups][D][12][RW];
  __shared__ __align__(16) Cx<R> gsh[kQGroups][kGrp];
  __shared__ int stab[kTMax];  // slot of every time
  const Geom& g = A.g;
  for (int i = threadIdx.x; i < g.tp; i += blockDim.x) stab[i] = slot_of(g, i);
  __syncthreads();
  const int q = threadIdx.x, r = q % kGrp, gi = q / kGrp;
  const unsigned mask = 0xFFFFu << (q & 16);
  const size_t grp = (size_t)blockIdx.x * kQGroups + gi;
  if (grp >= (size_t)A.nrhs * g.Nl) return;  // the group's 16 lanes leave together
  const int l = (int)(grp / A.nrhs), k = (int)(grp % A.nrhs);
  const int T = g.T, tp = g.tp;
  const bool act = r < 12;
  const int rc = act ? r : 0;  // lanes 12-15 address component 0 but never load or store
  const int sr = rc / 3, cr = rc - 3 * (rc / 3);
  const size_t base = ((size_t)k * g.Nl + l) * NSPIN_C * tp;
  const Cx<R>* in = A.in + base + (size_t)(A.swap_in ? (rc + 6) % 12 : rc) * tp;
  Cx<R>* out = A.out + base + (size_t)rc * tp;
  const Cx<R>* xp = A.xpost ? A.xpost + base + (size_t)rc * tp : nullptr;
  const Cx<R>* S = A.sinv + (size_t)l * T * kBlk + 12 * rc;  // lane rc's row: S[t * 144 + k]
  const Cx<R>* Zl = A.zv + (size_t)l * T * kBlk + 12 * rc;
  const Cx<R>* ut = AX ? nullptr : A.ut + (size_t)l * 9 * tp;
  Cx<R>(*rg)[12][RW] = ring[gi];
  Cx<R>* sh = gsh[gi];

  // forward sweep: z_t to out
  Cx<R> z = czero<R>();
  {
    auto issue = [&](int t) {  // step t: b_t, and for lanes 0-5 row rc of Sigma_{t-1}^-1
      if (t < T && act) {
        Cx<R>* d = rg[t % D][rc];
        cp_async<R>(d + 12, in + stab[t]);
        if (t >= 1 && r < 6) cp_row<R>(d, S + (size_t)(t - 1) * kBlk);
      }
      cp_commit();
    };
    for (int t = 0; t < D - 1; ++t) issue(t);
    for (int t = 0; t < T; ++t) {
      issue(t + D - 1);
      cp_wait<D - 1>();
      const Cx<R>* d = rg[t % D][rc];
      Cx<R> b = act ? d[12] : czero<R>();
      if (t > 0) {
        if (act) sh[rc] = z;
        __syncwarp(mask);
        const Cx<R> w = r < 6 ? row_dot(d, sh) : czero<R>();
        __syncwarp(mask);
        if (r < 6) sh[rc] = w;
        __syncwarp(mask);
        if (r < 6) {
          if (AX) {
            b = b + sh[rc];
          } else {  // + (W_{t-1}^dag w) on spin sr
            const int sl = stab[t - 1];
#pragma unroll
            for (int c = 0; c < 3; ++c) b = cfmaconj(b, ut[(size_t)(3 * c + cr) * tp + sl], sh[3 * sr + c]);
          }
        }
        __syncwarp(mask);
      }
      z = b;
      if (act) out[stab[t]] = z;
    }
    cp_wait<0>();
  }

  // backward sweep: chi_t to out
  Cx<R> y0 = czero<R>(), yT = czero<R>();
  {
    auto issue = [&](int u) {  // step u (t = N_t - 1 - u): row rc of Sigma_t^-1
      if (u < T && act) {
        cp_row<R>(rg[u % D][rc], S + (size_t)(T - 1 - u) * kBlk);
      }
      cp_commit();
    };
    for (int u = 0; u < D - 1; ++u) issue(u);
    Cx<R> zt = z;
    Cx<R> znext = act && T >= 2 ? out[stab[T - 2]] : czero<R>();
    Cx<R> y = czero<R>();
    for (int u = 0; u < T; ++u) {
      const int t = T - 1 - u;
      issue(u + D - 1);
      cp_wait<D - 1>();
      const Cx<R>* d = rg[u % D][rc];
      Cx<R> v = zt;
      zt = znext;
      if (act && t >= 2) znext = out[stab[t - 2]];  // used two steps on
      if (u > 0) {  // + [P_- (x) W_t] y_{t+1}
        if (act) sh[rc] = y;
        __syncwarp(mask);
        if (act && r >= 6) {
          if (AX) {
            v = v + sh[rc];
          } else {
            const int sl = stab[t];
#pragma unroll
            for (int c = 0; c < 3; ++c) v = cfma(v, ut[(size_t)(3 * cr + c) * tp + sl], sh[3 * sr + c]);
          }
        }
        __syncwarp(mask);
      }
      if (act) sh[rc] = v;
      __syncwarp(mask);
      y = act ? row_dot(d, sh) : czero<R>();
      __syncwarp(mask);
      if (act) out[stab[t]] = y;
      if (t == 0) y0 = y;
      if (t == T - 1) yT = y;
    }
    cp_wait<0>();
  }

  // c = Lambda W^dag chi (W^dag chi: the P_+ half of chi_{N_t-1}, the P_- half of chi_0)
  if (act) sh[rc] = r < 6 ? yT : y0;
  __syncwarp(mask);
  Cx<R> c = czero<R>();
  if (act) c = row_times(A.lam + (size_t)l * kBlk, rc, sh);
  __syncwarp(mask);
  if (act) sh[rc] = c;
  __syncwarp(mask);
  Cx<R> cv[12];
#pragma unroll
  for (int kk = 0; kk < 12; ++kk) cv[kk] = sh[kk];
  __syncwarp(mask);

  // out_t = xpost_t + apost (chi_t - Z_t c): independent steps
  {
    const bool post = xp != nullptr;
    auto issue = [&](int t) {  // step t: row rc of Z_t, and xpost_t
      if (t < T && act) {
        Cx<R>* d = rg[t % D][rc];
        cp_row<R>(d, Zl + (size_t)t * kBlk);
        if (post) cp_async<R>(d + 12, xp + stab[t]);
      }
      cp_commit();
    };
    for (int t = 0; t < D - 1; ++t) issue(t);
    Cx<R> ct = act ? out[stab[0]] : czero<R>();
    Cx<R> cnext = act && T >= 2 ? out[stab[1]] : czero<R>();
    for (int t = 0; t < T; ++t) {
      issue(t + D - 1);
      cp_wait<D - 1>();
      const Cx<R>* d = rg[t % D][rc];
      Cx<R> x = ct;
      ct = cnext;
      if (act && t + 2 < T) cnext = out[stab[t + 2]];
      if (act) {
        x = x - row_dot_reg(d, cv);
        out[stab[t]] = post ? d[12] + A.apost * x : x;
      }
    }
    cp_wait<0>();
  }
  if (act)
    for (int t = T; t < tp; ++t) out[stab[t]] = czero<R>();  // padding slots stay zero
}

// The same Q^-1 for four or more sources: a CTA holds kQGroups consecutive sources of one line,
// which read the same block rows, so one ring serves all its groups. The first group's lanes fill
// it D - 1 steps ahead; a CTA barrier per step publishes a slot to every group and also tells the
// filling lanes that the slot they refill next has been read. Each group's own operands (b_t,
// z_t, chi_t and the post-axpy operand) come from global memory two steps ahead in registers.
// Groups past the last source compute on zeros and store nothing, but join every barrier.
template <typename R, bool AX>
__global__ void __launch_bounds__(kQGroups * kGrp) k_qinv_apply_shared(const QinvArgs<R> A) {
  constexpr int D = QRing<R>::depth, RW = QRing<R>::row;
  __shared__ __align__(16) Cx<R> ring[D][12][RW];
  __shared__ __align__(16) Cx<R> gsh[kQGroups][kGrp];
  __shared__ int stab[kTMax];  // slot of every time
  const Geom& g = A.g;
  for (int i = threadIdx.x; i < g.tp; i += blockDim.x) stab[i] = slot_of(g, i);
  __syncthreads();
  const int q = threadIdx.x, r = q % kGrp, gi = q / kGrp;
  const unsigned mask = 0xFFFFu << (q & 16);
  const int nq = (A.nrhs + kQGroups - 1) / kQGroups;
  const int l = (int)(blockIdx.x / nq), k = (int)(blockIdx.x % nq) * kQGroups + gi;
  const int T = g.T, tp = g.tp;
  const bool act = r < 12;
  const bool io = act && k < A.nrhs;   // lanes that load and store this group's source
  const bool fill = act && gi == 0;    // lanes that fill the ring
  const int rc = act ? r : 0;
  const int sr = rc / 3, cr = rc - 3 * (rc / 3);
  const size_t base = ((size_t)(k < A.nrhs ? k : 0) * g.Nl + l) * NSPIN_C * tp;
  const Cx<R>* in = A.in + base + (size_t)(A.swap_in ? (rc + 6) % 12 : rc) * tp;
  Cx<R>* out = A.out + base + (size_t)rc * tp;
  const Cx<R>* xp = A.xpost ? A.xpost + base + (size_t)rc * tp : nullptr;
  const Cx<R>* S = A.sinv + (size_t)l * T * kBlk + 12 * rc;
  const Cx<R>* Zl = A.zv + (size_t)l * T * kBlk + 12 * rc;
  const Cx<R>* ut = AX ? nullptr : A.ut + (size_t)l * 9 * tp;
  Cx<R>* sh = gsh[gi];
  auto ld = [&](const Cx<R>* p, int t) { return io && t < T ? p[stab[t]] : czero<R>(); };

  // forward sweep: z_t to out
  Cx<R> z = czero<R>();
  {
    auto issue = [&](int t) {  // step t: rows 0-5 of Sigma_{t-1}^-1
      if (fill && r < 6 && t >= 1 && t < T) cp_row<R>(ring[t % D][rc], S + (size_t)(t - 1) * kBlk);
      if (gi == 0) cp_commit();
    };
    for (int t = 0; t < D - 1; ++t) issue(t);
    Cx<R> bt = ld(in, 0), bn = ld(in, 1);
    for (int t = 0; t < T; ++t) {
      if (gi == 0) cp_wait<D - 2>();
      __syncthreads();
      issue(t + D - 1);
      const Cx<R>* d = ring[t % D][rc];
      Cx<R> b = bt;
      bt = bn;
      bn = ld(in, t + 2);
      if (t > 0) {
        if (act) sh[rc] = z;
        __syncwarp(mask);
        const Cx<R> w = r < 6 ? row_dot(d, sh) : czero<R>();
        __syncwarp(mask);
        if (r < 6) sh[rc] = w;
        __syncwarp(mask);
        if (r < 6) {
          if (AX) {
            b = b + sh[rc];
          } else {
            const int sl = stab[t - 1];
#pragma unroll
            for (int c = 0; c < 3; ++c) b = cfmaconj(b, ut[(size_t)(3 * c + cr) * tp + sl], sh[3 * sr + c]);
          }
        }
        __syncwarp(mask);
      }
      z = b;
      if (io) out[stab[t]] = z;
    }
    if (gi == 0) cp_wait<0>();
    __syncthreads();
  }

  // backward sweep: chi_t to out
  Cx<R> y0 = czero<R>(), yT = czero<R>();
  {
    auto issue = [&](int u) {  // step u (t = N_t - 1 - u): row rc of Sigma_t^-1
      if (fill && u < T) cp_row<R>(ring[u % D][rc], S + (size_t)(T - 1 - u) * kBlk);
      if (gi == 0) cp_commit();
    };
    for (int u = 0; u < D - 1; ++u) issue(u);
    Cx<R> zt = z;
    Cx<R> zn = ld(out, T - 2);
    Cx<R> y = czero<R>();
    for (int u = 0; u < T; ++u) {
      const int t = T - 1 - u;
      if (gi == 0) cp_wait<D - 2>();
      __syncthreads();
      issue(u + D - 1);
      const Cx<R>* d = ring[u % D][rc];
      Cx<R> v = zt;
      zt = zn;
      zn = t >= 2 ? ld(out, t - 2) : czero<R>();
      if (u > 0) {
        if (act) sh[rc] = y;
        __syncwarp(mask);
        if (act && r >= 6) {
          if (AX) {
            v = v + sh[rc];
          } else {
            const int sl = stab[t];
#pragma unroll
            for (int c = 0; c < 3; ++c) v = cfma(v, ut[(size_t)(3 * cr + c) * tp + sl], sh[3 * sr + c]);
          }
        }
        __syncwarp(mask);
      }
      if (act) sh[rc] = v;
      __syncwarp(mask);
      y = act ? row_dot(d, sh) : czero<R>();
      __syncwarp(mask);
      if (io) out[stab[t]] = y;
      if (t == 0) y0 = y;
      if (t == T - 1) yT = y;
    }
    if (gi == 0) cp_wait<0>();
    __syncthreads();
  }

  // c = Lambda W^dag chi
  if (act) sh[rc] = r < 6 ? yT : y0;
  __syncwarp(mask);
  Cx<R> c = czero<R>();
  if (act) c = row_times(A.lam + (size_t)l * kBlk, rc, sh);
  __syncwarp(mask);
  if (act) sh[rc] = c;
  __syncwarp(mask);
  Cx<R> cv[12];
#pragma unroll
  for (int kk = 0; kk < 12; ++kk) cv[kk] = sh[kk];
  __syncwarp(mask);

  // out_t = xpost_t + apost (chi_t - Z_t c)
  {
    auto issue = [&](int t) {  // step t: row rc of Z_t
      if (fill && t < T) cp_row<R>(ring[t % D][rc], Zl + (size_t)t * kBlk);
      if (gi == 0) cp_commit();
    };
    for (int t = 0; t < D - 1; ++t) issue(t);
    Cx<R> ct = ld(out, 0), cn = ld(out, 1);
    Cx<R> xt = xp ? ld(xp, 0) : czero<R>(), xn = xp ? ld(xp, 1) : czero<R>();
    for (int t = 0; t < T; ++t) {
      if (gi == 0) cp_wait<D - 2>();
      __syncthreads();
      issue(t + D - 1);
      const Cx<R>* d = ring[t % D][rc];
      Cx<R> x = ct, xv = xt;
      ct = cn;
      cn = ld(out, t + 2);
      if (xp) {
        xt = xn;
        xn = ld(xp, t + 2);
      }
      x = x - row_dot_reg(d, cv);
      if (io) out[stab[t]] = xp ? xv + A.apost * x : x;
    }
    if (gi == 0) cp_wait<0>();
  }
  if (io)
    for (int t = T; t < tp; ++t) out[stab[t]] = czero<R>();  // padding slots stay zero
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
template <typename R>
struct QFactors {
  const Cx<R>* sinv[2];
  const Cx<R>* lam[2];
  const Cx<R>* zv[2];
};

const char* const kSinvName[2][2] = {{"fsw_sinv0_f64", "fsw_sinv1_f64"}, {"fsw_sinv0_f32", "fsw_sinv1_f32"}};
const char* const kLamName[2][2] = {{"fsw_lam0_f64", "fsw_lam1_f64"}, {"fsw_lam0_f32", "fsw_lam1_f32"}};
const char* const kZName[2][2] = {{"fsw_z0_f64", "fsw_z1_f64"}, {"fsw_z0_f32", "fsw_z1_f32"}};

template <typename R>
const Cx<R>* gauge_ut(wf_handle* h, int p) {
  if constexpr (sizeof(R) == 8)
    return h->ut64[p].as<Cx<double>>();
  else
    return h->ut32[p].as<Cx<float>>();
}
template <typename R>
const Cx<R>* gauge_pl(wf_handle* h, int p) {
  if constexpr (sizeof(R) == 8)
    return h->pl64[p].as<Cx<double>>();
  else
    return h->pl32[p].as<Cx<float>>();
}
template <typename R>
const Cx<R>* gauge_us(wf_handle* h, int p) {
  if constexpr (sizeof(R) == 8)
    return h->us64[p].as<Cx<double>>();
  else
    return h->us32[p].as<Cx<float>>();
}
template <typename R>
const Cx<R>* clover_of(wf_handle* h, int p) {
  if constexpr (sizeof(R) == 8)
    return h->clov64[p].as<Cx<double>>();
  else
    return h->clov32[p].as<Cx<float>>();
}
template <typename R>
const char* tag(const char* f64, const char* f32) {
  return sizeof(R) == 8 ? f64 : f32;
}


// The finalizer of Steele, Lea and Flood's SplitMix64 generator, a 64-bit mixing function
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// *out += sum over words i of mix64(w_i + (i + 1) golden + salt) (mod 2^64): a fingerprint of the
// n words that does not depend on the order in which threads add their parts
__global__ void __launch_bounds__(256) k_fingerprint(const unsigned long long* __restrict__ w, size_t n,
                                                     unsigned long long salt, unsigned long long* out) {
  unsigned long long acc = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += mix64(w[i] + (i + 1) * 0x9e3779b97f4a7c15ull + salt);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Whether the factors of precision R on the handle were formed from the gauge field and clover
// term it holds now. The factors depend on the frame, the presence of a clover term and the
// arrays the setup reads (clover blocks, U_t or P of both parities); a 64-bit fingerprint of those
// is kept beside the factors, and *key receives the current one.
template <typename R>
bool qinv_current(wf_handle* h, unsigned long long* key) {
  const Geom& g = h->g;
  cudaStream_t s = h->stream;
  unsigned long long* kb = h->buf<unsigned long long>(tag<R>("fsw_key_f64", "fsw_key_f32"), 3);
  WF_CUDA(cudaMemsetAsync(kb, 0, sizeof(unsigned long long), s));
  auto add = [&](const void* p, size_t bytes, unsigned long long salt) {
    const size_t n = bytes / sizeof(unsigned long long);
    const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8));
    Prof P(h, "fsw_fingerprint");
    k_fingerprint<<<blocks, 256, 0, s>>>(static_cast<const unsigned long long*>(p), n, salt, kb);
    WF_CUDA(cudaGetLastError());
  };
  for (int p = 0; p < 2; ++p) {
    if (h->clover) add(clover_of<R>(h, p), (size_t)g.Nl * 72 * g.tp * sizeof(Cx<R>), 0x1000ull + p);
    if (h->axial)
      add(gauge_pl<R>(h, p), (size_t)g.Nl * 9 * sizeof(Cx<R>), 0x2000ull + p);
    else
      add(gauge_ut<R>(h, p), (size_t)g.Nl * 9 * g.tp * sizeof(Cx<R>), 0x3000ull + p);
  }
  unsigned long long hk[3];
  WF_CUDA(cudaMemcpyAsync(hk, kb, sizeof(hk), cudaMemcpyDeviceToHost, s));
  WF_CUDA(cudaStreamSynchronize(s));
  *key = hk[0] ^ (h->axial ? 0x5bd1e995ull : 0ull) ^ (h->clover ? 0xc2b2ae35ull << 32 : 0ull);
  return hk[2] == 1 && hk[1] == *key;
}

// Record (valid = 1) or withdraw (valid = 0) the fingerprint of the factors of precision R
template <typename R>
void qinv_mark(wf_handle* h, unsigned long long key, unsigned long long valid) {
  unsigned long long* kb = h->buf<unsigned long long>(tag<R>("fsw_key_f64", "fsw_key_f32"), 3);
  const unsigned long long v[2] = {key, valid};
  WF_CUDA(cudaMemcpyAsync(kb + 1, v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
  WF_CUDA(cudaStreamSynchronize(h->stream));
}

// Factor T_0 and form Lambda on every line of both parities from the handle's gauge field and
// clover term (A = 0 without one), in precision R from the gauge and clover copies of that
// precision; kept until the gauge field, the clover term or the frame changes.
template <typename R>
void qinv_setup(wf_handle* h) {
  unsigned long long key = 0;
  if (qinv_current<R>(h, &key)) return;
  qinv_mark<R>(h, key, 0);  // a factorisation that fails part-way leaves no valid mark
  const Geom& g = h->g;
  cudaStream_t s = h->stream;
  const int w = sizeof(R) == 8 ? 0 : 1;
  const size_t nb = (size_t)g.Nl * g.T * kBlk, nl = (size_t)g.Nl * kBlk;
  const size_t per_line = (size_t)12 * g.T * 12 * sizeof(Cx<R>);
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)g.Nl, kScratchBytes / per_line));
  Cx<R>* scratch = h->buf<Cx<R>>(tag<R>("fsw_scratch_f64", "fsw_scratch_f32"), (size_t)chunk * 12 * g.T * 12);
  int* singular = h->buf<int>("fsw_singular", 1);
  WF_CUDA(cudaMemsetAsync(singular, 0, sizeof(int), s));
  for (int p = 0; p < 2; ++p) {
    SetupArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.g = g;
    a.H = h->clover ? clover_of<R>(h, p) : nullptr;
    a.ut = gauge_ut<R>(h, p);
    a.pl = gauge_pl<R>(h, p);
    a.s = (R)g.bc;
    a.sinv = h->buf<Cx<R>>(kSinvName[w][p], nb);
    a.lam = h->buf<Cx<R>>(kLamName[w][p], nl);
    a.zv = h->buf<Cx<R>>(kZName[w][p], nb);
    a.scratch = scratch;
    a.singular = singular;
    for (int l0 = 0; l0 < g.Nl; l0 += chunk) {
      a.line0 = l0;
      const int lines = std::min(chunk, g.Nl - l0);
      Prof P(h, tag<R>("qinv_setup_f64", "qinv_setup_f32"));
      if (h->axial)
        k_qinv_setup<R, true><<<lines, kSetupThreads, 0, s>>>(a);
      else
        k_qinv_setup<R, false><<<lines, kSetupThreads, 0, s>>>(a);
      WF_CUDA(cudaGetLastError());
    }
  }
  int sing = 0;
  WF_CUDA(cudaMemcpyAsync(&sing, singular, sizeof(int), cudaMemcpyDeviceToHost, s));
  WF_CUDA(cudaStreamSynchronize(s));
  if (sing) throw Error(WF_ESINGULAR, "a block of mu + A - D_t on a time line has no inverse");
  qinv_mark<R>(h, key, 1);
}

template <typename R>
QFactors<R> qfactors(wf_handle* h) {
  const Geom& g = h->g;
  const int w = sizeof(R) == 8 ? 0 : 1;
  QFactors<R> f;
  for (int p = 0; p < 2; ++p) {
    f.sinv[p] = h->buf<Cx<R>>(kSinvName[w][p], (size_t)g.Nl * g.T * kBlk);
    f.lam[p] = h->buf<Cx<R>>(kLamName[w][p], (size_t)g.Nl * kBlk);
    f.zv[p] = h->buf<Cx<R>>(kZName[w][p], (size_t)g.Nl * g.T * kBlk);
  }
  return f;
}

// out = xpost + apost Q^-1 (S) in on the lines of parity p
template <typename R>
void qinv(wf_handle* h, const QFactors<R>& F, int p, const Cx<R>* in, Cx<R>* out, int nrhs, int swap_in = 0,
          const Cx<R>* xpost = nullptr, double apost = 0.0) {
  QinvArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.g = h->g;
  a.nrhs = nrhs;
  a.in = in;
  a.out = out;
  a.xpost = xpost;
  a.apost = (R)apost;
  a.swap_in = swap_in;
  a.sinv = F.sinv[p];
  a.lam = F.lam[p];
  a.zv = F.zv[p];
  a.ut = gauge_ut<R>(h, p);
  a.pl = gauge_pl<R>(h, p);
  a.s = (R)h->g.bc;
  if (h->g.tp > kTMax) throw Error(WF_EINVAL, "Q^-1 kernel: padded time line longer than 256 slots");
  const size_t groups = (size_t)nrhs * h->g.Nl;
  const unsigned blocks = (unsigned)((groups + kQGroups - 1) / kQGroups);
  Prof P(h, tag<R>("qinv_apply_f64", "qinv_apply_f32"));
  if (nrhs >= kQGroups) {  // one ring per CTA of kQGroups sources of one line
    const unsigned sblocks = (unsigned)((size_t)h->g.Nl * ((nrhs + kQGroups - 1) / kQGroups));
    if (h->axial)
      k_qinv_apply_shared<R, true><<<sblocks, kQGroups * kGrp, 0, h->stream>>>(a);
    else
      k_qinv_apply_shared<R, false><<<sblocks, kQGroups * kGrp, 0, h->stream>>>(a);
  } else if (h->axial) {
    k_qinv_apply<R, true><<<blocks, kQGroups * kGrp, 0, h->stream>>>(a);
  } else {
    k_qinv_apply<R, false><<<blocks, kQGroups * kGrp, 0, h->stream>>>(a);
  }
  WF_CUDA(cudaGetLastError());
}

// out = xpost + apost (S) D_s in on the lines of parity p (in: the other parity)
template <typename R>
void hop(wf_handle* h, int p, const Cx<R>* in, Cx<R>* out, int nrhs, const Cx<R>* xpost = nullptr,
         double apost = 0.0, int swap_out = 0) {
  LineArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.g = h->g;
  a.parity = p;
  a.nrhs = nrhs;
  a.src = SRC_HOP;
  a.opu = OP_COPY;
  a.opl = OP_COPY;
  a.src_up = in;
  a.src_lo = in + 6 * h->g.tp;
  a.ut = gauge_ut<R>(h, p);
  a.pl = gauge_pl<R>(h, p);
  a.us_out = gauge_us<R>(h, p);
  a.us_nbr = gauge_us<R>(h, 1 - p);
  a.inv_mu = (R)(1.0 / h->g.mu);
  a.bc = (R)h->g.bc;
  a.xpost = xpost;
  a.apost = (R)apost;
  a.swap_out = swap_out;
  a.out = out;
  a.drop_job = -1;
  Prof P(h, tag<R>("fsw_hop_f64", "fsw_hop_f32"));
  launch_line<R>(a, LK_GENERIC, h->axial, h->stream);
}

// M-hat_full (dagger: its adjoint) on internal odd fields x -> out; e1, e2 (even) and o1 (odd) are
// work fields of the size of x
template <typename R>
void schur_full(wf_handle* h, const QFactors<R>& F, const Cx<R>* x, Cx<R>* out, int dagger, int nrhs, Cx<R>* e1,
                Cx<R>* e2, Cx<R>* o1) {
  const double m = -1.0 / (h->g.gamma_f * h->g.gamma_f);
  if (!dagger) {
    hop<R>(h, 0, x, e1, nrhs);                          // D_s^eo x
    qinv<R>(h, F, 0, e1, e2, nrhs);                     // (Q^ee)^-1
    hop<R>(h, 1, e2, o1, nrhs);                         // D_s^oe
    qinv<R>(h, F, 1, o1, out, nrhs, 0, x, m);           // x - gamma_f^-2 (Q^oo)^-1 ...
  } else {
    qinv<R>(h, F, 1, x, o1, nrhs, 1);                   // (Q^oo)^-1 S x
    hop<R>(h, 0, o1, e1, nrhs);
    qinv<R>(h, F, 0, e1, e2, nrhs);
    hop<R>(h, 1, e2, out, nrhs, x, m, 1);               // x - gamma_f^-2 S D_s^oe ...
  }
}

// ----------------------------------------------------------------------------
// C-ABI bodies
// ----------------------------------------------------------------------------
const Cx<double>* stage_in(wf_handle* h, const double* p, size_t elems, const char* name) {
  if (!p) throw Error(WF_EINVAL, "null array argument");
  if (device_resident(p, h->device)) return reinterpret_cast<const Cx<double>*>(p);
  Cx<double>* d = h->buf<Cx<double>>(name, elems);
  WF_CUDA(cudaMemcpyAsync(d, p, elems * sizeof(Cx<double>), cudaMemcpyHostToDevice, h->stream));
  return d;
}
Cx<double>* stage_out(wf_handle* h, double* p, size_t elems, const char* name, bool& staged) {
  if (!p) throw Error(WF_EINVAL, "null array argument");
  staged = !device_resident(p, h->device);
  return staged ? h->buf<Cx<double>>(name, elems) : reinterpret_cast<Cx<double>*>(p);
}
void finish(wf_handle* h, double* p, const Cx<double>* d, size_t elems, bool staged) {
  if (staged) WF_CUDA(cudaMemcpyAsync(p, d, elems * sizeof(Cx<double>), cudaMemcpyDeviceToHost, h->stream));
  WF_CUDA(cudaStreamSynchronize(h->stream));
}
void check_handle(wf_handle* h, int nrhs) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (nrhs < 1 || nrhs > WF_MAX_SOLVE_RHS) throw Error(WF_EINVAL, "nrhs must lie in [1, WF_MAX_SOLVE_RHS]");
}

template <typename R>
int apply_qinv_abi(wf_handle* h, const double* in, double* out, int nrhs) {
  check_handle(h, nrhs);
  const Geom& g = h->g;
  const size_t le = h->lex_elems() * nrhs, nt = h->half_int() * nrhs;
  const Cx<double>* din = stage_in(h, in, le, "stage_in");
  bool staged;
  Cx<double>* dout = stage_out(h, out, le, "stage_out", staged);
  Cx<R>* ie = h->buf<Cx<R>>(tag<R>("fsw_ie_f64", "fsw_ie_f32"), nt);
  Cx<R>* io = h->buf<Cx<R>>(tag<R>("fsw_io_f64", "fsw_io_f32"), nt);
  Cx<R>* oe = h->buf<Cx<R>>(tag<R>("fsw_oe_f64", "fsw_oe_f32"), nt);
  Cx<R>* oo = h->buf<Cx<R>>(tag<R>("fsw_oo_f64", "fsw_oo_f32"), nt);
  qinv_setup<R>(h);
  const QFactors<R> F = qfactors<R>(h);
  {
    Prof P(h, tag<R>("import_spinor_f64", "import_spinor_f32"));
    launch_import_spinor<R>(g, din, ie, io, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), h->stream);
  }
  qinv<R>(h, F, 0, ie, oe, nrhs);
  qinv<R>(h, F, 1, io, oo, nrhs);
  {
    Prof P(h, tag<R>("export_spinor_f64", "export_spinor_f32"));
    launch_export_spinor<R>(g, oe, oo, dout, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), h->stream);
  }
  finish(h, out, dout, le, staged);
  return WF_OK;
}

template <typename R>
int apply_schur_full_abi(wf_handle* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  check_handle(h, nrhs);
  const Geom& g = h->g;
  const size_t ce = (size_t)nrhs * g.T * g.Nl * NSPIN_C, nt = h->half_int() * nrhs;
  const Cx<double>* din = stage_in(h, in_odd, ce, "stage_in");
  bool staged;
  Cx<double>* dout = stage_out(h, out_odd, ce, "stage_out", staged);
  Cx<R>* x = h->buf<Cx<R>>(tag<R>("fsw_x_f64", "fsw_x_f32"), nt);
  Cx<R>* o = h->buf<Cx<R>>(tag<R>("fsw_o_f64", "fsw_o_f32"), nt);
  Cx<R>* e1 = h->buf<Cx<R>>(tag<R>("fsw_e1_f64", "fsw_e1_f32"), nt);
  Cx<R>* e2 = h->buf<Cx<R>>(tag<R>("fsw_e2_f64", "fsw_e2_f32"), nt);
  Cx<R>* o1 = h->buf<Cx<R>>(tag<R>("fsw_o1_f64", "fsw_o1_f32"), nt);
  qinv_setup<R>(h);
  const QFactors<R> F = qfactors<R>(h);
  {
    Prof P(h, tag<R>("import_compact_f64", "import_compact_f32"));
    launch_import_compact<R>(g, din, x, nrhs, 0, frame_rot(h, 1), h->stream);
  }
  schur_full<R>(h, F, x, o, dagger, nrhs, e1, e2, o1);
  {
    Prof P(h, tag<R>("export_compact_f64", "export_compact_f32"));
    launch_export_compact<R>(g, o, dout, nrhs, 0, frame_rot(h, 1), h->stream);
  }
  finish(h, out_odd, dout, ce, staged);
  return WF_OK;
}

// r_p = eta_p - (M + A) psi on parity p, FP64 (the true residual of M_SW)
void msw_residual(wf_handle* h, int p, const Cx<double>* psi_e, const Cx<double>* psi_o, const Cx<double>* eta,
                  Cx<double>* r, int nrhs) {
  MArgs<double> a;
  std::memset(&a, 0, sizeof(a));
  a.g = h->g;
  a.parity = p;
  a.nrhs = nrhs;
  a.psi_p = p ? psi_o : psi_e;
  a.psi_q = p ? psi_e : psi_o;
  a.ut = h->ut64[p].as<Cx<double>>();
  a.pl = h->pl64[p].as<Cx<double>>();
  a.us_out = h->us64[p].as<Cx<double>>();
  a.us_nbr = h->us64[1 - p].as<Cx<double>>();
  a.x = eta;
  a.a = -1.0;
  a.out = r;
  a.mu = h->g.mu;
  a.inv_gf = 1.0 / h->g.gamma_f;
  a.bc = h->g.bc;
  {
    Prof P(h, "apply_M_f64");
    launch_apply_M<double>(a, h->axial, h->stream);
  }
  if (h->clover) {
    Prof P(h, "clover_apply_f64");
    launch_clover_apply<double>(h->g, h->clov64[p].as<Cx<double>>(), a.psi_p, r, r, -1.0, nrhs, h->stream);
  }
}

// Per-rhs |x_e|^2 + |x_o|^2 to the host
void norms(wf_handle* h, const Cx<double>* xe, const Cx<double>* xo, int nrhs, std::vector<double>& out) {
  const size_t n = h->half_int();
  double* partial = h->buf<double>("fsw_partial", 1024 * (size_t)nrhs);
  double* nn = h->buf<double>("fsw_norms", 2 * (size_t)nrhs);
  {
    Prof P(h, "norm2_f64", 4);
    launch_norm2<double>(xe, n, nrhs, partial, nn, h->stream);
    launch_norm2<double>(xo, n, nrhs, partial, nn + nrhs, h->stream);
  }
  std::vector<double> hn(2 * (size_t)nrhs);
  WF_CUDA(cudaMemcpyAsync(hn.data(), nn, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  WF_CUDA(cudaStreamSynchronize(h->stream));
  out.resize(nrhs);
  for (int k = 0; k < nrhs; ++k) out[k] = hn[k] + hn[nrhs + k];
}

// CGNR on M-hat_full y = b in precision R, from y = 0, each right-hand side k to
// |b - M-hat y| <= rho[k] |b| (rho[k] >= 1 or b = 0: no iteration); stops at `left` iterations.
// its[k] gains the iterations right-hand side k took; returns the iterations of the loop.
template <typename R>
int cgnr_full(wf_handle* h, const QFactors<R>& F, const Cx<R>* b, Cx<R>* y, int nrhs, const std::vector<double>& rho,
              int left, std::vector<int>& its) {
  cudaStream_t s = h->stream;
  const size_t n = h->half_int(), nt = n * nrhs;
  Cx<R>* r = h->buf<Cx<R>>(tag<R>("fsw_cg_r_f64", "fsw_cg_r_f32"), nt);
  Cx<R>* p = h->buf<Cx<R>>(tag<R>("fsw_cg_p_f64", "fsw_cg_p_f32"), nt);
  Cx<R>* q = h->buf<Cx<R>>(tag<R>("fsw_cg_q_f64", "fsw_cg_q_f32"), nt);
  Cx<R>* sv = h->buf<Cx<R>>(tag<R>("fsw_cg_s_f64", "fsw_cg_s_f32"), nt);
  Cx<R>* e1 = h->buf<Cx<R>>(tag<R>("fsw_e1_f64", "fsw_e1_f32"), nt);
  Cx<R>* e2 = h->buf<Cx<R>>(tag<R>("fsw_e2_f64", "fsw_e2_f32"), nt);
  Cx<R>* o1 = h->buf<Cx<R>>(tag<R>("fsw_o1_f64", "fsw_o1_f32"), nt);
  double* sc = h->buf<double>("fsw_cg_scalars", 5 * (size_t)nrhs);
  double *gam = sc, *gnew = sc + nrhs, *qq = sc + 2 * nrhs, *rr = sc + 3 * nrhs, *bb = sc + 4 * nrhs;
  int* active = h->buf<int>("fsw_cg_active", nrhs);
  double* partial = h->buf<double>("fsw_partial", 1024 * (size_t)nrhs);
  WF_CUDA(cudaMemsetAsync(y, 0, nt * sizeof(Cx<R>), s));
  WF_CUDA(cudaMemcpyAsync(r, b, nt * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, s));
  schur_full<R>(h, F, r, sv, 1, nrhs, e1, e2, o1);
  WF_CUDA(cudaMemcpyAsync(p, sv, nt * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, s));
  {
    Prof P(h, tag<R>("norm2_f64", "norm2_f32"), 4);
    launch_norm2<R>(sv, n, nrhs, partial, gam, s);
    launch_norm2<R>(b, n, nrhs, partial, bb, s);
  }
  std::vector<double> hb(nrhs), hr(nrhs);
  std::vector<int> act(nrhs);
  WF_CUDA(cudaMemcpyAsync(hb.data(), bb, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  WF_CUDA(cudaStreamSynchronize(s));
  int nact = 0;
  for (int k = 0; k < nrhs; ++k) {
    if (!std::isfinite(hb[k])) throw Error(WF_ENAN, "NaN or Inf in the preconditioned source");
    act[k] = hb[k] > 0.0 && rho[k] < 1.0 ? 1 : 0;
    nact += act[k];
  }
  WF_CUDA(cudaMemcpyAsync(active, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
  int it = 0;
  while (nact > 0 && it < left) {
    schur_full<R>(h, F, p, q, 0, nrhs, e1, e2, o1);
    {
      Prof P(h, tag<R>("norm2_f64", "norm2_f32"), 2);
      launch_norm2<R>(q, n, nrhs, partial, qq, s);
    }
    {
      Prof P(h, tag<R>("cg_xr_f64", "cg_xr_f32"), 2);
      launch_cg_xr<R>(y, r, p, q, n, nrhs, gam, qq, active, partial, rr, s);
    }
    ++it;
    for (int k = 0; k < nrhs; ++k) its[k] += act[k];
    WF_CUDA(cudaMemcpyAsync(hr.data(), rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    WF_CUDA(cudaStreamSynchronize(s));
    nact = 0;
    for (int k = 0; k < nrhs; ++k) {
      if (!act[k]) continue;
      if (!std::isfinite(hr[k])) throw Error(WF_ENAN, "NaN or Inf in a CG residual");
      if (hr[k] <= rho[k] * rho[k] * hb[k]) act[k] = 0;
      nact += act[k];
    }
    WF_CUDA(cudaMemcpyAsync(active, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
    if (nact == 0) break;
    schur_full<R>(h, F, r, sv, 1, nrhs, e1, e2, o1);
    {
      Prof P(h, tag<R>("norm2_f64", "norm2_f32"), 2);
      launch_norm2<R>(sv, n, nrhs, partial, gnew, s);
    }
    {
      Prof P(h, tag<R>("cg_p_f64", "cg_p_f32"), 2);
      launch_cg_p<R>(p, sv, n, nrhs, gnew, gam, active, s);
      launch_copy_scalar(gam, gnew, nrhs, s, active);
    }
  }
  return it;
}

// M_SW psi = eta with full SW temporal preconditioning and 3-D Schur, by defect correction: every
// pass solves M_SW delta = r in precision R (source preparation (Q^oo)^-1 (r_o + gamma_f^-1 D_s^oe
// (Q^ee)^-1 r_e), CGNR on M-hat_full, reconstruction delta_e = (Q^ee)^-1 (r_e + gamma_f^-1 D_s^eo
// delta_o)), adds delta to psi in FP64 and recomputes the FP64 true residual r = eta - M_SW psi.
template <typename R>
int solve_full_abi(wf_handle* h, const double* rhs, double* x, int nrhs, double tol, int* iters_out,
                   double* resid_out) {
  check_handle(h, nrhs);
  if (!(tol > 0)) throw Error(WF_EINVAL, "tol must be > 0");
  const Geom& g = h->g;
  cudaStream_t s = h->stream;
  const size_t le = h->lex_elems() * nrhs, n = h->half_int(), nt = n * nrhs;
  const Cx<double>* drhs = stage_in(h, rhs, le, "stage_in");
  bool staged;
  Cx<double>* dx = stage_out(h, x, le, "stage_out", staged);
  Cx<double>* eta_e = h->buf<Cx<double>>("fsw_eta_e", nt);
  Cx<double>* eta_o = h->buf<Cx<double>>("fsw_eta_o", nt);
  Cx<double>* psi_e = h->buf<Cx<double>>("fsw_psi_e", nt);
  Cx<double>* psi_o = h->buf<Cx<double>>("fsw_psi_o", nt);
  Cx<double>* r_e = h->buf<Cx<double>>("fsw_r_e", nt);
  Cx<double>* r_o = h->buf<Cx<double>>("fsw_r_o", nt);
  Cx<R>* re = h->buf<Cx<R>>(tag<R>("fsw_re_f64", "fsw_re_f32"), nt);
  Cx<R>* ro = h->buf<Cx<R>>(tag<R>("fsw_ro_f64", "fsw_ro_f32"), nt);
  Cx<R>* ue = h->buf<Cx<R>>(tag<R>("fsw_ue_f64", "fsw_ue_f32"), nt);
  Cx<R>* wo = h->buf<Cx<R>>(tag<R>("fsw_wo_f64", "fsw_wo_f32"), nt);
  Cx<R>* bo = h->buf<Cx<R>>(tag<R>("fsw_bo_f64", "fsw_bo_f32"), nt);
  Cx<R>* yo = h->buf<Cx<R>>(tag<R>("fsw_yo_f64", "fsw_yo_f32"), nt);
  Cx<R>* we = h->buf<Cx<R>>(tag<R>("fsw_we_f64", "fsw_we_f32"), nt);
  qinv_setup<R>(h);
  const QFactors<R> F = qfactors<R>(h);
  {
    Prof P(h, "import_spinor_f64");
    launch_import_spinor<double>(g, drhs, eta_e, eta_o, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), s);
  }
  WF_CUDA(cudaMemsetAsync(psi_e, 0, nt * sizeof(Cx<double>), s));
  WF_CUDA(cudaMemsetAsync(psi_o, 0, nt * sizeof(Cx<double>), s));
  WF_CUDA(cudaMemcpyAsync(r_e, eta_e, nt * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, s));
  WF_CUDA(cudaMemcpyAsync(r_o, eta_o, nt * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, s));
  std::vector<double> etan, rn;
  norms(h, eta_e, eta_o, nrhs, etan);
  for (int k = 0; k < nrhs; ++k)
    if (!std::isfinite(etan[k])) throw Error(WF_ENAN, "NaN or Inf in the source");
  rn = etan;
  const double gi = 1.0 / g.gamma_f;
  // each pass aims at half the target; an FP32 pass at no less than 1e-5 of its source
  const double floor = sizeof(R) == 4 ? 1e-5 : 0.0;
  std::vector<double> rho(nrhs), rel(nrhs, 1.0);
  std::vector<int> its(nrhs, 0);
  int used = 0;
  bool done = false;
  for (int pass = 0; pass < 8 && !done; ++pass) {
    if constexpr (sizeof(R) == 8) {
      WF_CUDA(cudaMemcpyAsync(re, r_e, nt * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, s));
      WF_CUDA(cudaMemcpyAsync(ro, r_o, nt * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, s));
    } else {
      Prof P(h, "d2f", 2);
      launch_d2f(r_e, re, nt, s);
      launch_d2f(r_o, ro, nt, s);
    }
    for (int k = 0; k < nrhs; ++k) {
      rel[k] = etan[k] > 0 ? std::sqrt(rn[k] / etan[k]) : 0.0;
      rho[k] = rel[k] <= tol ? 1.0 : std::max(floor, 0.5 * tol / rel[k]);
      if (rel[k] <= tol) {  // converged: a zero source keeps its solution as it is
        WF_CUDA(cudaMemsetAsync(re + k * n, 0, n * sizeof(Cx<R>), s));
        WF_CUDA(cudaMemsetAsync(ro + k * n, 0, n * sizeof(Cx<R>), s));
      }
    }
    qinv<R>(h, F, 0, re, ue, nrhs);                   // (Q^ee)^-1 r_e
    hop<R>(h, 1, ue, wo, nrhs, ro, gi);               // r_o + gamma_f^-1 D_s^oe ...
    qinv<R>(h, F, 1, wo, bo, nrhs);                   // b = (Q^oo)^-1 ...
    used += cgnr_full<R>(h, F, bo, yo, nrhs, rho, std::max(1, h->maxiter - used), its);
    hop<R>(h, 0, yo, we, nrhs, re, gi);               // r_e + gamma_f^-1 D_s^eo delta_o
    qinv<R>(h, F, 0, we, ue, nrhs);                   // delta_e
    if constexpr (sizeof(R) == 8) {
      Prof P(h, "axpby_f64", 2);
      launch_axpby<double>(psi_e, ue, nt, 1.0, 1.0, s);
      launch_axpby<double>(psi_o, yo, nt, 1.0, 1.0, s);
    } else {
      Prof P(h, "add_f_to_d", 2);
      launch_add_f_to_d(psi_e, ue, nt, s);
      launch_add_f_to_d(psi_o, yo, nt, s);
    }
    msw_residual(h, 0, psi_e, psi_o, eta_e, r_e, nrhs);
    msw_residual(h, 1, psi_e, psi_o, eta_o, r_o, nrhs);
    norms(h, r_e, r_o, nrhs, rn);
    done = true;
    for (int k = 0; k < nrhs; ++k) {
      if (!std::isfinite(rn[k])) throw Error(WF_ENAN, "NaN or Inf in a true residual");
      rel[k] = etan[k] > 0 ? std::sqrt(rn[k] / etan[k]) : 0.0;
      if (rel[k] > tol) done = false;
    }
    if (used >= h->maxiter) break;
  }
  {
    Prof P(h, "export_spinor_f64");
    launch_export_spinor<double>(g, psi_e, psi_o, dx, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), s);
  }
  finish(h, x, dx, le, staged);
  for (int k = 0; k < nrhs; ++k) {
    if (iters_out) iters_out[k] = its[k];
    if (resid_out) resid_out[k] = rel[k];
  }
  return done ? WF_OK : WF_ENOCONV;
}

template <typename F>
int guard(wf_handle* h, F&& f) {
  if (!h) return WF_EINVAL;
  h->err.clear();
  try {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) WF_CUDA(cudaSetDevice(h->device));
    return f();
  } catch (const Error& e) {
    h->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return WF_ENOMEM;
  } catch (const std::exception& e) {
    h->err = e.what();
    return WF_ECUDA;
  } catch (...) {
    h->err = "unknown error";
    return WF_ECUDA;
  }
}

}  // namespace
}  // namespace wf

using namespace wf;

extern "C" {

int wf_apply_Qinv(wf_handle_t* h, const double* in, double* out, int nrhs) {
  return guard(h, [&]() { return apply_qinv_abi<double>(h, in, out, nrhs); });
}
int wf_apply_Qinv_f32(wf_handle_t* h, const double* in, double* out, int nrhs) {
  return guard(h, [&]() { return apply_qinv_abi<float>(h, in, out, nrhs); });
}
int wf_apply_schur_full_sw(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  return guard(h, [&]() { return apply_schur_full_abi<double>(h, in_odd, out_odd, dagger ? 1 : 0, nrhs); });
}
int wf_apply_schur_full_sw_f32(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  return guard(h, [&]() { return apply_schur_full_abi<float>(h, in_odd, out_odd, dagger ? 1 : 0, nrhs); });
}
int wf_solve_full_sw(wf_handle_t* h, const double* rhs, double* x, int nrhs, double tol, int precision,
                     int* iters_out, double* true_resid_out) {
  return guard(h, [&]() {
    if (precision == WF_FP64) return solve_full_abi<double>(h, rhs, x, nrhs, tol, iters_out, true_resid_out);
    if (precision == WF_FP32) return solve_full_abi<float>(h, rhs, x, nrhs, tol, iters_out, true_resid_out);
    throw Error(WF_EINVAL, "precision must be WF_FP64 or WF_FP32");
  });
}

}  // extern "C"
