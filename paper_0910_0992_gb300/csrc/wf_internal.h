// Host-side internals of libwf: the handle, device buffers and kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "wf_common.cuh"

namespace wf {

// Error carried from a failing step up to the C-ABI boundary (never crosses it).
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define WF_CUDA(call)                                                                           \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      throw ::wf::Error(3 /*WF_ECUDA*/, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

// Owning device allocation (cudaMalloc / cudaFree), zero-filled on allocation.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // make sure at least nbytes are held; contents are zero after a (re)allocation
  void ensure(size_t nbytes, cudaStream_t s) {
    if (nbytes <= bytes) return;
    release();
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
      p = nullptr;
      throw Error(2 /*WF_ENOMEM*/, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    bytes = nbytes;
    WF_CUDA(cudaMemsetAsync(p, 0, nbytes, s));
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

// ----------------------------------------------------------------------------
// Launchers (defined in the .cu files)
// ----------------------------------------------------------------------------
template <typename R> struct LineArgs;

// which compiled variant of the line kernel to launch: the three Schur-operator kernels
// have their source and solve ops fixed at compile time; LK_GENERIC reads them from the
// arguments
enum LineKind { LK_GENERIC = 0, LK_SCHUR_A = 1, LK_SCHUR_B = 2, LK_SCHUR_C = 3 };

template <typename R>
void launch_line(const LineArgs<R>& a, int kind, bool axial, cudaStream_t s);

// one launch (or one per kMaxLattices) over a ragged batch of lattices, each with its own
// arguments: K-a, K-b or K-c on the line kernel (n sites per lane), and K-b / K-c on the
// one-thread-per-site kernel (tables attached; 128-slot lattices and the others launch apart)
template <typename R>
void launch_line_multi(const std::vector<LineArgs<R>>& as, int kind, cudaStream_t s);
template <typename R>
void launch_line_wide_multi(const std::vector<LineArgs<R>>& as, int kind, cudaStream_t s);

// axial-frame line kernels with one thread per time site (wf_wide.cu), same arguments
bool wide_supported(const Geom& g);
template <typename R>
void launch_line_wide(const LineArgs<R>& a, int kind, cudaStream_t s);

// bulk-copy-fed FP32 axial hop kernels K-b / K-c for 128-slot lines (wf_pipe.cu): gsrc sources per
// unit (1 or 2), ns shared-memory stages (2..4); units: [nunits] (first source, line) pairs in
// traversal order; err: device error word, set when a bounded wait expired
bool pipe_supported(const Geom& g);
void launch_hop_pipe(const LineArgs<float>& a, int kind, int gsrc, int ns, const int2* units, int nunits, int* err,
                     cudaStream_t s);

// TMA-fed FP32 axial variant of the Schur hop kernels (wf_tma.cu); err: device error word
bool tma_supported(const Geom& g);
void launch_line_tma(const LineArgs<float>& a, int kind, int* err, cudaStream_t s);

template <typename R>
struct MArgs {
  Geom g;
  int parity;
  int nrhs;
  const Cx<R>* psi_p;  // own parity  [nrhs][Nl][12][tp]
  const Cx<R>* psi_q;  // other parity
  const Cx<R>* ut;     // U_t of the own parity (general frame)
  const Cx<R>* pl;     // per-line boundary link P (axial frame)
  const Cx<R>* us_out; // forward spatial links, own parity
  const Cx<R>* us_nbr; // forward spatial links, other parity
  const Cx<R>* x;      // out = x + a * (M psi) if x != nullptr
  R a;
  int swap;            // read psi and write the result with the spin halves exchanged (M^dag = S M S)
  Cx<R>* out;
  R mu, inv_gf, bc;
};
template <typename R>
void launch_apply_M(const MArgs<R>& a, bool axial, cudaStream_t s);
// the long-line variants (lines of 129 to 256 slots; wf_kernels_long_f32.cu, wf_kernels_long_f64.cu)
template <typename R>
void launch_line_long(const LineArgs<R>& a, int kind, bool axial, cudaStream_t s);
template <typename R>
void launch_apply_M_long(const MArgs<R>& a, bool axial, cudaStream_t s);

// layout conversions
// g_e / g_o (or gr): per-parity colour rotations of the axial frame, [l][9][tp] FP64, or null
template <typename R>
void launch_import_spinor(const Geom& g, const Cx<double>* lex, Cx<R>* even, Cx<R>* odd, int nrhs, int g5,
                          const Cx<double>* g_e, const Cx<double>* g_o, cudaStream_t s);
template <typename R>
void launch_export_spinor(const Geom& g, const Cx<R>* even, const Cx<R>* odd, Cx<double>* lex, int nrhs, int g5,
                          const Cx<double>* g_e, const Cx<double>* g_o, cudaStream_t s);
template <typename R>
void launch_import_compact(const Geom& g, const Cx<double>* cmp, Cx<R>* half, int nrhs, int g5, const Cx<double>* gr,
                           cudaStream_t s);
template <typename R>
void launch_export_compact(const Geom& g, const Cx<R>* half, Cx<double>* cmp, int nrhs, int g5, const Cx<double>* gr,
                           cudaStream_t s);
void launch_import_gauge(const Geom& g, const Cx<double>* lex, Cx<double>* ut[2], Cx<double>* us[2],
                         cudaStream_t s);
void launch_tline_init(const Geom& g, const Cx<double>* ut, Cx<double>* lamb, Cx<double>* lamf, int* singular,
                       cudaStream_t s);
void launch_axial_frame(const Geom& g, Cx<double>* ut_to_g, Cx<double>* pl, Cx<double>* lamb, Cx<double>* wrap,
                        int* singular, cudaStream_t s);
void launch_rotate_links(const Geom& g, Cx<double>* us[2], const Cx<double>* gg[2], cudaStream_t s);
// flag |= 1 if a link of the lexicographic field U ([nlinks][3][3]) is not finite, |= 2 if one is
// not SU(3) within tol (entries of U^dag U - 1 and det U - 1)
void launch_check_links(const Cx<double>* U, size_t nlinks, double tol, int* flag, cudaStream_t s);
void launch_d2f(const Cx<double>* in, Cx<float>* out, size_t n, cudaStream_t s);
// FP32 copy of spatial links in their two-row storage (nlinks = 3 Nl per parity)
void launch_d2f_links(const Cx<double>* in, Cx<float>* out, size_t nlinks, int tp, cudaStream_t s);
void launch_f2d(const Cx<float>* in, Cx<double>* out, size_t n, cudaStream_t s);

// BLAS-1 on flat [nrhs][n] arrays; scalars live in device memory. offs (ragged batches of several
// lattices): device prefix table [nrhs + 1] of each rhs's first element in the packed vectors, n
// then only sizes the grid (the largest length); null: rhs k occupies [k n, (k + 1) n).
template <typename R>
void launch_norm2(const Cx<R>* x, size_t n, int nrhs, double* partial, double* out, cudaStream_t s,
                  const size_t* offs = nullptr);
// CG updates: launch_cg_xr does r -= alpha q (alpha = gamma / qq) with |r|^2 into rr_out, and
// x += alpha p unless x is null; then upd (if given) records the right-hand sides that took the
// update. launch_cg_p does p = s + beta p (beta = gamma_new / gamma_old) for the active ones and,
// with x given, first the deferred x += alpha p (alpha = gamma_old / qq) for those flagged in upd.
template <typename R>
void launch_cg_xr(Cx<R>* x, Cx<R>* r, const Cx<R>* p, const Cx<R>* q, size_t n, int nrhs, const double* gamma,
                  const double* qq, const int* active, double* partial, double* rr_out, cudaStream_t s,
                  const size_t* offs = nullptr, int* upd = nullptr);
template <typename R>
void launch_cg_p(Cx<R>* p, const Cx<R>* sv, size_t n, int nrhs, const double* gamma_new, const double* gamma_old,
                 const int* active, cudaStream_t s, const size_t* offs = nullptr, Cx<R>* x = nullptr,
                 const double* qq = nullptr, const int* upd = nullptr);
template <typename R>
void launch_axpby(Cx<R>* y, const Cx<R>* x, size_t n, double a, double b, cudaStream_t s);  // y = a x + b y
void launch_add_f_to_d(Cx<double>* y, const Cx<float>* x, size_t n, cudaStream_t s);      // y += x
// FP16-stored CG vectors (Cx16, wf_line.cuh), stored divided by a per-rhs scale sigma
struct Cx16;
void launch_norm2_h16(const Cx16* x, size_t n, int nrhs, double* partial, double* out, cudaStream_t s);
void launch_cg_xr_h16(Cx<float>* x, Cx16* r, const Cx16* p, const Cx16* q, size_t n, int nrhs, const double* gamma,
                      const double* qq, const double* sigma, const int* active, double* partial, double* rr_out,
                      cudaStream_t s);
void launch_cg_p_h16(Cx16* p, const Cx16* sv, size_t n, int nrhs, const double* gnew, const double* gold,
                     const int* active, cudaStream_t s);
template <typename T>  // T = Cx<double>, Cx<float> or Cx16: out = in * f[rhs]
void launch_scale_to_h16(Cx16* out, const T* in, size_t n, int nrhs, const double* f, cudaStream_t s);
void launch_sub_d_f(Cx<float>* out, const Cx<double>* r64, const Cx<float>* a, size_t n, cudaStream_t s);  // out = r64 - a
void launch_scale_from_h16(Cx<float>* out, const Cx16* in, size_t n, int nrhs, const double* f, cudaStream_t s);
void launch_copy_scalar(double* dst, const double* src, int nrhs, cudaStream_t s, const int* active = nullptr);
void launch_cg_check(const double* rr, int* active, int* state, int* iters, const double* tgt2, const double* ru2,
                     int nrhs, cudaStream_t s);

// 4-D even-odd comparator (wf_eo4d.cu)
template <typename R>
struct EoArgs {
  Geom g;
  int par;          // 4-D parity of the output sites
  int nrhs;
  const Cx<R>* in;  // field of the other parity, [rhs][L^3][12][T/2]
  // out = a * D_w in + b1 * x1 + b2 * x2 (x1, x2 of the output parity; null = absent)
  const Cx<R>* x1;
  R b1;
  const Cx<R>* x2;
  R b2;
  R a;
  int swap_in, swap_out;  // read / write the P_+ and P_- spin halves exchanged (gamma_5 up to sign)
  int stream_out;         // store with the evict-first cache policy (the result is not read again soon)
  int df;                 // R = double only: compute in double-float (FP64 storage, FP32 arithmetic)
  Cx<R>* out;
  double* norm2;          // if set: atomically add |out|^2 per rhs
  const Cx<R>* ut[2];     // general frame: U_t per 3-D parity, line layout
  const Cx<R>* pl[2];     // axial frame: boundary link P per line
  const Cx<R>* us[2];     // spatial forward links per 3-D parity, line layout
  R inv_gf, bc;
};
template <typename R>
void launch_dslash4(const EoArgs<R>& a, bool axial, cudaStream_t s);
// compact_par < 0: full lexicographic fields; 0 / 1: arrays of the sites of that 4-D parity only
template <typename R>
void launch_import_eo(const Geom& g, const Cx<double>* lex, Cx<R>* even, Cx<R>* odd, int nrhs, const Cx<double>* g0,
                      const Cx<double>* g1, int compact_par, cudaStream_t s);
template <typename R>
void launch_export_eo(const Geom& g, const Cx<R>* even, const Cx<R>* odd, Cx<double>* lex, int nrhs,
                      const Cx<double>* g0, const Cx<double>* g1, int compact_par, cudaStream_t s);

// pseudofermion force: link outer products (wf_force.cu)
struct ForceArgs {
  Geom g;
  int parity;  // 3-D parity of the links' base sites
  bool axial;
  // temporal: C_L pair (a, b) and C_R pair (c, e), fields of this parity [Nl][12][tp]
  const Cx<double>* a;
  const Cx<double>* b;
  const Cx<double>* c;
  const Cx<double>* e;
  // spatial: Q uses w (this parity) and v (other parity, at x + k); R uses vr (this parity)
  // and wr (other parity, at x + k)
  const Cx<double>* w;
  const Cx<double>* v;
  const Cx<double>* vr;
  const Cx<double>* wr;
  const Cx<double>* ut;      // general frame: U_t [Nl][9][tp]; axial frame: rotation g
  const Cx<double>* pl;      // axial frame: P per line
  const Cx<double>* us_p;    // spatial links of this parity (frame of the solve)
  double coef;               // 2 / gamma_f^2
  double bc;
  double* F;                 // [V][4][8], caller's gauge
};
void launch_force(const ForceArgs& a, cudaStream_t s);

// Clover term (wf_clover.cu): build H_a, H_b (half the chiral blocks of A, [Nl][2][36][tp] per
// parity) from the lexicographic FP64 links, rotated by rot[p] (the axial-frame rotation, or
// null in the caller's gauge); F_scratch holds V x 6 matrices
void launch_clover_build(const Geom& g, const Cx<double>* U_lex, const Cx<double>* rot[2], double c_s, double c_t,
                         Cx<double>* F_scratch, Cx<double>* H[2], cudaStream_t s);
// out = acc + alpha A in on one parity (acc may be null; padding slots get acc or zero)
template <typename R>
void launch_clover_apply(const Geom& g, const Cx<R>* H, const Cx<R>* in, Cx<R>* out, const Cx<R>* acc, double alpha,
                         int nrhs, cudaStream_t s);
// the same on a 4-D even-odd field [rhs][L^3][12][T/2] with blocks [L^3][2][36][T/2]
template <typename R>
void launch_clover_apply_eo(const Geom& g, const Cx<R>* H, const Cx<R>* in, Cx<R>* out, const Cx<R>* acc,
                            double alpha, int nrhs, cudaStream_t s);
// blocks of mu + A and of (mu + A)^-1 (halved) in the 4-D even-odd layout, per 4-D parity, from
// the line-layout blocks H; *singular set where mu + A has no inverse
void launch_clover_eo4_build(const Geom& g, const Cx<double>* H[2], Cx<double>* M[2], Cx<double>* Minv[2],
                             int* singular, cudaStream_t s);
// out = in with the spin halves exchanged, n elements of [..][12][tp] fields
template <typename R>
void launch_swap_halves(const Cx<R>* in, Cx<R>* out, size_t n, int tp, cudaStream_t s);

}  // namespace wf
