// BLAS-1 for the Krylov loop: norms with FP64 accumulation and the fused CG vector
// updates. Arrays are [nrhs][n] complex; per-RHS scalars live in device memory, so
// the CG loop runs without host round trips.
#include "wf_internal.h"
#include "wf_line.cuh"

namespace wf {

constexpr int kBT = 256;
constexpr int kMaxPartial = 1024;  // partial sums per RHS (scratch: nrhs * kMaxPartial doubles)

static int parts_for(size_t n) {
  size_t b = (n + (size_t)kBT * 8 - 1) / ((size_t)kBT * 8);
  if (b < 1) b = 1;
  if (b > kMaxPartial) b = kMaxPartial;
  return (int)b;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kBT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = 0.0;
  if (threadIdx.x < kBT / 32) v = red[threadIdx.x];
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// Ragged batches (several lattices in one CG): offs, if set, is the prefix table [nrhs + 1] of the
// right-hand sides' first elements in the packed vectors (then n only sizes the grid).
__device__ __forceinline__ void rhs_range(int rhs, size_t n, const size_t* offs, size_t& off, size_t& len) {
  if (offs) {
    off = offs[rhs];
    len = offs[rhs + 1] - off;
  } else {
    off = (size_t)rhs * n;
    len = n;
  }
}

template <typename R>
__global__ void __launch_bounds__(kBT) k_norm2(const Cx<R>* __restrict__ x, size_t n, double* partial,
                                               const size_t* offs) {
  const int rhs = blockIdx.y;
  size_t o0, len;
  rhs_range(rhs, n, offs, o0, len);
  n = len;
  const Cx<R>* xr = x + o0;
  R part = R(0);  // per-thread partial sum in the field's precision; FP64 across threads
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    const Cx<R> v = xr[i];
    part = fma(v.re, v.re, fma(v.im, v.im, part));
  }
  double acc = block_sum((double)part);
  if (threadIdx.x == 0) partial[rhs * gridDim.x + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kBT) k_final_sum(const double* __restrict__ partial, int parts, double* out) {
  const int rhs = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < parts; i += kBT) acc += partial[rhs * parts + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[rhs] = acc;
}

template <typename R>
void launch_norm2(const Cx<R>* x, size_t n, int nrhs, double* partial, double* out, cudaStream_t s,
                  const size_t* offs) {
  const int parts = parts_for(n);
  k_norm2<R><<<dim3(parts, nrhs), kBT, 0, s>>>(x, n, partial, offs);
  k_final_sum<<<nrhs, kBT, 0, s>>>(partial, parts, out);
  WF_CUDA(cudaGetLastError());
}
template void launch_norm2<float>(const Cx<float>*, size_t, int, double*, double*, cudaStream_t, const size_t*);
template void launch_norm2<double>(const Cx<double>*, size_t, int, double*, double*, cudaStream_t, const size_t*);

// alpha = gamma / |q|^2; x += alpha p (x null: left to k_cg_p, see below); r -= alpha q; partial
// |r|^2; upd (if given) records which right-hand sides took this update
template <typename R>
__global__ void __launch_bounds__(kBT) k_cg_xr(Cx<R>* __restrict__ x, Cx<R>* __restrict__ r, const Cx<R>* __restrict__ p,
                                                const Cx<R>* __restrict__ q, size_t n, const double* gamma,
                                                const double* qq, const int* active, double* partial,
                                                const size_t* offs, int* upd) {
  const int rhs = blockIdx.y;
  const bool on = active[rhs] != 0;
  const double qn = qq[rhs];
  const R alpha = (on && qn > 0.0) ? (R)(gamma[rhs] / qn) : R(0);
  if (upd && blockIdx.x == 0 && threadIdx.x == 0) upd[rhs] = on ? 1 : 0;
  size_t off, len;
  rhs_range(rhs, n, offs, off, len);
  n = len;
  R part = R(0);  // per-thread partial |r|^2 in the field's precision; FP64 across threads
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    const Cx<R> qv = q[off + i];
    Cx<R> rv = r[off + i];
    if (x) {
      const Cx<R> pv = p[off + i];
      Cx<R> xv = x[off + i];
      xv.re = fma(alpha, pv.re, xv.re);
      xv.im = fma(alpha, pv.im, xv.im);
      x[off + i] = xv;
    }
    rv.re = fma(-alpha, qv.re, rv.re);
    rv.im = fma(-alpha, qv.im, rv.im);
    r[off + i] = rv;
    part = fma(rv.re, rv.re, fma(rv.im, rv.im, part));
  }
  double acc = block_sum((double)part);
  if (threadIdx.x == 0) partial[rhs * gridDim.x + blockIdx.x] = acc;
}

template <typename R>
void launch_cg_xr(Cx<R>* x, Cx<R>* r, const Cx<R>* p, const Cx<R>* q, size_t n, int nrhs, const double* gamma,
                  const double* qq, const int* active, double* partial, double* rr_out, cudaStream_t s,
                  const size_t* offs, int* upd) {
  const int parts = parts_for(n);
  k_cg_xr<R><<<dim3(parts, nrhs), kBT, 0, s>>>(x, r, p, q, n, gamma, qq, active, partial, offs, upd);
  k_final_sum<<<nrhs, kBT, 0, s>>>(partial, parts, rr_out);
  WF_CUDA(cudaGetLastError());
}
template void launch_cg_xr<float>(Cx<float>*, Cx<float>*, const Cx<float>*, const Cx<float>*, size_t, int,
                                  const double*, const double*, const int*, double*, double*, cudaStream_t,
                                  const size_t*, int*);
template void launch_cg_xr<double>(Cx<double>*, Cx<double>*, const Cx<double>*, const Cx<double>*, size_t, int,
                                   const double*, const double*, const int*, double*, double*, cudaStream_t,
                                   const size_t*, int*);

// beta = gamma_new / gamma_old; p = s + beta p for the active right-hand sides. With x given, the
// x update that k_cg_xr left out happens here, before p changes: x += alpha p with alpha =
// gamma_old / qq for the right-hand sides that took this iteration's r update (upd), also those
// that stopped at it. One pass over p then serves both updates.
template <typename R>
__global__ void __launch_bounds__(kBT) k_cg_p(Cx<R>* __restrict__ p, const Cx<R>* __restrict__ sv, size_t n,
                                               const double* gnew, const double* gold, const int* active,
                                               const size_t* offs, Cx<R>* __restrict__ x, const double* qq,
                                               const int* upd) {
  const int rhs = blockIdx.y;
  const bool on = active[rhs] != 0;
  const bool dox = x && upd[rhs];
  if (!on && !dox) return;
  const double go = gold[rhs];
  const R beta = go > 0.0 ? (R)(gnew[rhs] / go) : R(0);
  const double qn = dox ? qq[rhs] : 0.0;
  const R alpha = qn > 0.0 ? (R)(go / qn) : R(0);
  size_t off, len;
  rhs_range(rhs, n, offs, off, len);
  n = len;
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    Cx<R> pv = p[off + i];
    if (dox) {
      Cx<R> xv = x[off + i];
      xv.re = fma(alpha, pv.re, xv.re);
      xv.im = fma(alpha, pv.im, xv.im);
      x[off + i] = xv;
    }
    if (on) {
      const Cx<R> s = sv[off + i];
      pv.re = fma(beta, pv.re, s.re);
      pv.im = fma(beta, pv.im, s.im);
      p[off + i] = pv;
    }
  }
}

template <typename R>
void launch_cg_p(Cx<R>* p, const Cx<R>* sv, size_t n, int nrhs, const double* gnew, const double* gold,
                 const int* active, cudaStream_t s, const size_t* offs, Cx<R>* x, const double* qq, const int* upd) {
  const int parts = parts_for(n) * 2;
  k_cg_p<R><<<dim3(parts, nrhs), kBT, 0, s>>>(p, sv, n, gnew, gold, active, offs, x, qq, upd);
  WF_CUDA(cudaGetLastError());
}
template void launch_cg_p<float>(Cx<float>*, const Cx<float>*, size_t, int, const double*, const double*,
                                 const int*, cudaStream_t, const size_t*, Cx<float>*, const double*, const int*);
template void launch_cg_p<double>(Cx<double>*, const Cx<double>*, size_t, int, const double*, const double*,
                                  const int*, cudaStream_t, const size_t*, Cx<double>*, const double*, const int*);

template <typename R>
__global__ void __launch_bounds__(kBT) k_axpby(Cx<R>* __restrict__ y, const Cx<R>* __restrict__ x, size_t n, R a, R b) {
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    const Cx<R> xv = x[i];
    Cx<R> yv = y[i];
    yv.re = a * xv.re + b * yv.re;
    yv.im = a * xv.im + b * yv.im;
    y[i] = yv;
  }
}
template <typename R>
void launch_axpby(Cx<R>* y, const Cx<R>* x, size_t n, double a, double b, cudaStream_t s) {
  k_axpby<R><<<parts_for(n) * 2, kBT, 0, s>>>(y, x, n, (R)a, (R)b);
  WF_CUDA(cudaGetLastError());
}
template void launch_axpby<float>(Cx<float>*, const Cx<float>*, size_t, double, double, cudaStream_t);
template void launch_axpby<double>(Cx<double>*, const Cx<double>*, size_t, double, double, cudaStream_t);

__global__ void __launch_bounds__(kBT) k_add_f_to_d(Cx<double>* __restrict__ y, const Cx<float>* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    Cx<double> yv = y[i];
    yv.re += (double)x[i].re;
    yv.im += (double)x[i].im;
    y[i] = yv;
  }
}
void launch_add_f_to_d(Cx<double>* y, const Cx<float>* x, size_t n, cudaStream_t s) {
  k_add_f_to_d<<<parts_for(n) * 2, kBT, 0, s>>>(y, x, n);
  WF_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------
// FP16-stored CG vectors (Cx16, one half2 per complex). Each right-hand side's vectors are
// stored divided by a scale sigma[rhs] that the solver resets at every reliable update, so that
// they stay O(1) in FP16; norms are of the stored (scaled) values, in FP32 per thread and FP64
// across threads.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float2 h16_ld(const Cx16* p, size_t i) { return __half22float2(p[i].v); }
__device__ __forceinline__ void h16_st(Cx16* p, size_t i, float re, float im) { p[i].v = __floats2half2_rn(re, im); }

__global__ void __launch_bounds__(kBT) k_norm2_h16(const Cx16* __restrict__ x, size_t n, double* partial) {
  const int rhs = blockIdx.y;
  const Cx16* xr = x + (size_t)rhs * n;
  float part = 0.f;
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    const float2 v = h16_ld(xr, i);
    part = fmaf(v.x, v.x, fmaf(v.y, v.y, part));
  }
  double acc = block_sum((double)part);
  if (threadIdx.x == 0) partial[rhs * gridDim.x + blockIdx.x] = acc;
}
void launch_norm2_h16(const Cx16* x, size_t n, int nrhs, double* partial, double* out, cudaStream_t s) {
  const int parts = parts_for(n);
  k_norm2_h16<<<dim3(parts, nrhs), kBT, 0, s>>>(x, n, partial);
  k_final_sum<<<nrhs, kBT, 0, s>>>(partial, parts, out);
  WF_CUDA(cudaGetLastError());
}

// alpha = gamma / |q|^2 (scaled units, so alpha is the true step); x += alpha sigma p (x in FP32,
// true units); r -= alpha q; partial |r|^2 (scaled)
__global__ void __launch_bounds__(kBT) k_cg_xr_h16(Cx<float>* __restrict__ x, Cx16* __restrict__ r,
                                                    const Cx16* __restrict__ p, const Cx16* __restrict__ q, size_t n,
                                                    const double* gamma, const double* qq, const double* sigma,
                                                    const int* active, double* partial) {
  const int rhs = blockIdx.y;
  // a stopped source keeps its vectors and its last partial norms (so the final sum repeats its
  // last |r|^2)
  if (!active[rhs]) return;
  const double qn = qq[rhs];
  const float alpha = qn > 0.0 ? (float)(gamma[rhs] / qn) : 0.f;
  const float ax = (float)(qn > 0.0 ? gamma[rhs] / qn * sigma[rhs] : 0.0);
  const size_t off = (size_t)rhs * n;
  float part = 0.f;
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    const float2 pv = h16_ld(p, off + i), qv = h16_ld(q, off + i);
    float2 rv = h16_ld(r, off + i);
    Cx<float> xv = x[off + i];
    xv.re = fmaf(ax, pv.x, xv.re);
    xv.im = fmaf(ax, pv.y, xv.im);
    rv.x = fmaf(-alpha, qv.x, rv.x);
    rv.y = fmaf(-alpha, qv.y, rv.y);
    x[off + i] = xv;
    h16_st(r, off + i, rv.x, rv.y);
    const float2 rs = h16_ld(r, off + i);  // the norm of what is stored
    part = fmaf(rs.x, rs.x, fmaf(rs.y, rs.y, part));
  }
  double acc = block_sum((double)part);
  if (threadIdx.x == 0) partial[rhs * gridDim.x + blockIdx.x] = acc;
}
void launch_cg_xr_h16(Cx<float>* x, Cx16* r, const Cx16* p, const Cx16* q, size_t n, int nrhs, const double* gamma,
                      const double* qq, const double* sigma, const int* active, double* partial, double* rr_out,
                      cudaStream_t s) {
  const int parts = parts_for(n);
  k_cg_xr_h16<<<dim3(parts, nrhs), kBT, 0, s>>>(x, r, p, q, n, gamma, qq, sigma, active, partial);
  k_final_sum<<<nrhs, kBT, 0, s>>>(partial, parts, rr_out);
  WF_CUDA(cudaGetLastError());
}

// beta = gamma_new / gamma_old; p = s + beta p
__global__ void __launch_bounds__(kBT) k_cg_p_h16(Cx16* __restrict__ p, const Cx16* __restrict__ sv, size_t n,
                                                   const double* gnew, const double* gold, const int* active) {
  const int rhs = blockIdx.y;
  if (!active[rhs]) return;
  const double go = gold[rhs];
  const float beta = go > 0.0 ? (float)(gnew[rhs] / go) : 0.f;
  const size_t off = (size_t)rhs * n;
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    const float2 sx = h16_ld(sv, off + i), pv = h16_ld(p, off + i);
    h16_st(p, off + i, fmaf(beta, pv.x, sx.x), fmaf(beta, pv.y, sx.y));
  }
}
void launch_cg_p_h16(Cx16* p, const Cx16* sv, size_t n, int nrhs, const double* gnew, const double* gold,
                     const int* active, cudaStream_t s) {
  k_cg_p_h16<<<dim3(parts_for(n) * 2, nrhs), kBT, 0, s>>>(p, sv, n, gnew, gold, active);
  WF_CUDA(cudaGetLastError());
}

// out = in * f[rhs] stored in FP16 (in: FP64, FP32 or FP16)
template <typename T>
__device__ __forceinline__ float2 ld_any(const T* p, size_t i) {
  if constexpr (std::is_same<T, Cx16>::value) {
    return h16_ld(p, i);
  } else {
    return make_float2((float)p[i].re, (float)p[i].im);
  }
}
// (in may be out: each element is read and written by one thread; FP32 arithmetic)
template <typename T>
__global__ void __launch_bounds__(kBT) k_scale_to_h16(Cx16* out, const T* in, size_t n, const double* f) {
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n;
  const float fr = (float)f[rhs];
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    const float2 v = ld_any(in, off + i);
    h16_st(out, off + i, v.x * fr, v.y * fr);
  }
}
template <typename T>
void launch_scale_to_h16(Cx16* out, const T* in, size_t n, int nrhs, const double* f, cudaStream_t s) {
  k_scale_to_h16<T><<<dim3(parts_for(n) * 2, nrhs), kBT, 0, s>>>(out, in, n, f);
  WF_CUDA(cudaGetLastError());
}
template void launch_scale_to_h16<Cx<double>>(Cx16*, const Cx<double>*, size_t, int, const double*, cudaStream_t);
template void launch_scale_to_h16<Cx<float>>(Cx16*, const Cx<float>*, size_t, int, const double*, cudaStream_t);
template void launch_scale_to_h16<Cx16>(Cx16*, const Cx16*, size_t, int, const double*, cudaStream_t);

// out (FP32) = in (FP16) * f[rhs]
__global__ void __launch_bounds__(kBT) k_scale_from_h16(Cx<float>* __restrict__ out, const Cx16* __restrict__ in,
                                                        size_t n, const double* f) {
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n;
  const float fr = (float)f[rhs];
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    const float2 v = h16_ld(in, off + i);
    out[off + i] = mk<float>(v.x * fr, v.y * fr);
  }
}
void launch_scale_from_h16(Cx<float>* out, const Cx16* in, size_t n, int nrhs, const double* f, cudaStream_t s) {
  k_scale_from_h16<<<dim3(parts_for(n) * 2, nrhs), kBT, 0, s>>>(out, in, n, f);
  WF_CUDA(cudaGetLastError());
}

// out = (float) r64 - a, the residual of an FP32 increment against the last FP64 residual
__global__ void __launch_bounds__(kBT) k_sub_d_f(Cx<float>* __restrict__ out, const Cx<double>* __restrict__ r64,
                                                  const Cx<float>* __restrict__ a, size_t n) {
  for (size_t i = blockIdx.x * (size_t)kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT) {
    const Cx<double> r = r64[i];
    const Cx<float> av = a[i];
    out[i] = mk<float>((float)r.re - av.re, (float)r.im - av.im);
  }
}
void launch_sub_d_f(Cx<float>* out, const Cx<double>* r64, const Cx<float>* a, size_t n, cudaStream_t s) {
  k_sub_d_f<<<parts_for(n) * 2, kBT, 0, s>>>(out, r64, a, n);
  WF_CUDA(cudaGetLastError());
}

// After the x, r update of a CG iteration, per right-hand side: count the iteration, stop a
// source whose residual met its target (state 1), stop and flag one whose residual fell below
// its reliable-update threshold (state 2: it waits for the host to recompute its residual)
__global__ void k_cg_check(const double* __restrict__ rr, int* __restrict__ active, int* __restrict__ state,
                           int* __restrict__ iters, const double* __restrict__ tgt2, const double* __restrict__ ru2,
                           int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || !active[k]) return;
  iters[k] += 1;
  if (rr[k] <= tgt2[k]) {
    active[k] = 0;
    state[k] = 1;
  } else if (rr[k] < ru2[k]) {
    active[k] = 0;
    state[k] = 2;
  }
}
void launch_cg_check(const double* rr, int* active, int* state, int* iters, const double* tgt2, const double* ru2,
                     int nrhs, cudaStream_t s) {
  k_cg_check<<<(nrhs + 127) / 128, 128, 0, s>>>(rr, active, state, iters, tgt2, ru2, nrhs);
  WF_CUDA(cudaGetLastError());
}

// dst = src for the active right-hand sides (all of them if active is null)
__global__ void k_copy_scalar(double* dst, const double* src, const int* active, int n) {
  int i = threadIdx.x;
  if (i < n && (!active || active[i])) dst[i] = src[i];
}
void launch_copy_scalar(double* dst, const double* src, int nrhs, cudaStream_t s, const int* active) {
  k_copy_scalar<<<1, 1024, 0, s>>>(dst, src, active, nrhs);
  WF_CUDA(cudaGetLastError());
}

}  // namespace wf
