// TMA-fed variant of the two hop kernels of the Schur operator (K-b, K-c), FP32, axial frame.
//
// In the line kernel the loads of the six hop directions are ordinary global loads whose data
// sits in registers until used, next to a 96-float accumulator, so only a few loads are in
// flight per warp and the kernel waits on memory. Here every operand of a direction is a
// contiguous block in HBM -- the neighbour line's P_+ and P_- spinor halves (6 tp complex each)
// and the link line in two-row storage (6 tp complex) -- and is brought into shared memory by
// one bulk asynchronous copy (cp.async.bulk, completion counted on an mbarrier). Each CTA is
// one warp working through its lines persistently with a two-stage ring: while a direction is
// computed from shared memory the next one is in flight, across line boundaries too, so the
// copies of the next line's first directions overlap the time-line scan of the current one.
// Shared memory reads are conflict-free (lane j reads slot m * 32 + j). Every wait is bounded:
// on expiry the kernel sets an error word, drains its outstanding copies (bounded as well) and
// returns; the host reports WF_ETIMEOUT. The expiry path is tested by skipping one copy on the
// host's request (environment WF_TEST_DROP_COPY=<job>), never by a fault.
#include <map>
#include <mutex>

#include "wf_internal.h"
#include "wf_line.cuh"

namespace wf {

namespace {

constexpr int kStages = 2;
// a wait gives up after this much device time (a copy normally lands within microseconds); the
// limit is on elapsed time because how long one try_wait may suspend is not specified
constexpr unsigned long long kWaitNs = 500000000ull;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the phase with the given parity of a barrier; false if kWaitNs passed first
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (!mbar_try_wait(bar, parity))
    if (now_ns() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  unsigned long long gsrc;
  asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(gsrc) : "l"(src));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// the axial time-line solve (wf_line.cuh) on the spin half starting at s0 of v
template <bool FWD>
__device__ __forceinline__ void solve_half_axial(Vec3<float> (&v)[NMAX][4], int s0, const LineArgs<float>& A, int l,
                                                 int jj) {
  Vec3<float> w[NMAX][2];
#pragma unroll
  for (int m = 0; m < NMAX; ++m) {
    w[m][0] = v[m][s0];
    w[m][1] = v[m][s0 + 1];
  }
  tline_solve_axial<float, 2, FWD>(w, A.pl + (size_t)l * 9, A.lamb + (size_t)l * 9, A.g, jj, A.inv_mu, A.bc);
#pragma unroll
  for (int m = 0; m < NMAX; ++m) {
    v[m][s0] = w[m][0];
    v[m][s0 + 1] = w[m][1];
  }
}

struct Stage {
  Cx<float>* up;
  Cx<float>* lo;
  Cx<float>* lk;
};

// the CTA's j-th line: lines lg = blockIdx.x + j * gridDim.x, rhs groups as in the line kernel
__device__ __forceinline__ void job_line(const LineArgs<float>& A, int lg, int& rhs, int& l) {
  line_rhs(lg, A.nrhs, A.g, rhs, l);
}

// issue the three bulk copies of direction d of line lg into stage st (lane 0 only)
__device__ __forceinline__ void issue(const LineArgs<float>& A, int lg, int d, const Stage& st, uint64_t* bar,
                                      int job) {
  if (job == A.drop_job && blockIdx.x == 0) return;  // injected fault: this stage never completes
  const Geom& g = A.g;
  const int tp = g.tp;
  int rhs, l;
  job_line(A, lg, rhs, l);
  int nb[6];
  neighbour_lines(g, A.parity, l, nb);
  const int k = d >> 1, ln = nb[d];
  constexpr int LNC = SpatialLinkNC<float>::value;
  const size_t sbase = ((size_t)rhs * g.Nl + ln) * NSPIN_C * tp;
  const Cx<float>* lk = (d & 1) == 0 ? A.us_out + ((size_t)k * g.Nl + l) * LNC * tp
                                     : A.us_nbr + ((size_t)k * g.Nl + ln) * LNC * tp;
  const unsigned half_bytes = 6u * tp * sizeof(Cx<float>);
  const unsigned link_bytes = (unsigned)LNC * tp * sizeof(Cx<float>);
  mbar_arrive_expect_tx(bar, 2 * half_bytes + link_bytes);
  bulk_copy_g2s(st.up, A.src_up + sbase, half_bytes, bar);
  bulk_copy_g2s(st.lo, A.src_lo + sbase, half_bytes, bar);
  bulk_copy_g2s(st.lk, lk, link_bytes, bar);
}

// one hop direction from shared memory into the accumulator (same arithmetic as hop_spatial)
__device__ __forceinline__ void hop_dir(Vec3<float> (&h)[NMAX][4], const Stage& st, int d, int tp, int n, int T,
                                        int jj) {
  const int k = d >> 1, dir = d & 1;
#pragma unroll
  for (int m = 0; m < NMAX; ++m) {
    if (m >= n || jj * n + m >= T) continue;
    const int sl = m * 32 + jj;
    Vec3<float> u0 = ldvec(st.up, tp, sl), u1 = ldvec(st.up + 3 * tp, tp, sl);
    Vec3<float> d0 = ldvec(st.lo, tp, sl), d1 = ldvec(st.lo + 3 * tp, tp, sl);
    Mat3<float> U = ldlink(st.lk, tp, sl);
    Vec3<float> s0, s1;
    isigma(k, d0, d1, s0, s1);
    Vec3<float> h0, h1;
    if (dir == 0) {
      h0 = vscale(0.5f, vadd(u0, s0));
      h1 = vscale(0.5f, vadd(u1, s1));
    } else {
      h0 = vscale(0.5f, vaxpy(-1.f, s0, u0));
      h1 = vscale(0.5f, vaxpy(-1.f, s1, u1));
    }
    Vec3<float> w0 = dir == 0 ? matvec(U, h0) : matvec_dag(U, h0);
    Vec3<float> w1 = dir == 0 ? matvec(U, h1) : matvec_dag(U, h1);
    h[m][0] = vadd(h[m][0], w0);
    h[m][1] = vadd(h[m][1], w1);
    Vec3<float> r0, r1;
    isigma(k, w0, w1, r0, r1);
    if (dir == 0) {
      h[m][2] = vaxpy(-1.f, r0, h[m][2]);
      h[m][3] = vaxpy(-1.f, r1, h[m][3]);
    } else {
      h[m][2] = vadd(h[m][2], r0);
      h[m][3] = vadd(h[m][3], r1);
    }
  }
}

template <int OPU, int OPL>
__global__ void __launch_bounds__(32) k_line_tma(const LineArgs<float> A, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Geom& g = A.g;
  const int tp = g.tp, n = g.n, T = g.T;
  const int jj = threadIdx.x;
  const size_t stage_elems = (size_t)18 * tp;  // up 6 tp, lo 6 tp, link 6 tp
  Stage st[kStages];
  for (int s = 0; s < kStages; ++s) {
    Cx<float>* b = reinterpret_cast<Cx<float>*>(smem) + s * stage_elems;
    st[s] = Stage{b, b + 6 * tp, b + 12 * tp};
  }
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * stage_elems * sizeof(Cx<float>));
  const int lines = A.nrhs * g.Nl;
  const int my_lines = blockIdx.x < lines ? (lines - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int jobs = my_lines * 6;
  if (jj == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  __syncwarp();
  if (jj == 0) {
    for (int j = 0; j < kStages && j < jobs; ++j) issue(A, blockIdx.x + (j / 6) * gridDim.x, j % 6, st[j], &bars[j], j);
  }
  unsigned phase[kStages] = {0u, 0u};
  bool failed = false;
  int job = 0;
  for (int li = 0; li < my_lines && !failed; ++li) {
    const int lg = blockIdx.x + li * gridDim.x;
    int rhs, l;
    job_line(A, lg, rhs, l);
    Vec3<float> v[NMAX][4];
#pragma unroll
    for (int m = 0; m < NMAX; ++m)
#pragma unroll
      for (int s = 0; s < 4; ++s) v[m][s] = vzero<float>();
    for (int d = 0; d < 6; ++d, ++job) {
      const int s = job % kStages;
      const bool ok = mbar_wait_bounded(&bars[s], phase[s]);
      // the decision is taken by the whole warp, so no lane is left behind at a __syncwarp
      if (__any_sync(0xffffffffu, !ok)) {
        failed = true;
        break;
      }
      phase[s] ^= 1u;
      hop_dir(v, st[s], d, tp, n, T, jj);
      __syncwarp();
      if (jj == 0 && job + kStages < jobs) {
        fence_proxy_async();
        const int nj = job + kStages;
        issue(A, blockIdx.x + (nj / 6) * gridDim.x, nj % 6, st[s], &bars[s], nj);
      }
    }
    if (failed) break;
    // time-line solves and store: the line kernel's epilogue
    const size_t base = ((size_t)rhs * g.Nl + l) * NSPIN_C * tp;
    if (OPU == OP_FWD) solve_half_axial<true>(v, 0, A, l, jj);
    if (OPL == OP_BWD) solve_half_axial<false>(v, 2, A, l, jj);
    float nrm = 0.f;
#pragma unroll
    for (int m = 0; m < NMAX; ++m) {
      if (m >= n) continue;
      const int sl = m * 32 + jj;
      const bool valid = jj * n + m < T;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int dh = A.swap_out ? 1 - h : h;
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
          const int comp0 = dh * 6 + s2 * 3;
          Vec3<float> val = valid ? v[m][2 * h + s2] : vzero<float>();
          if (A.xpost) val = vaxpy(A.apost, val, ldvec(A.xpost + base + comp0 * tp, tp, sl));
          stvec(A.out + base + comp0 * tp, tp, sl, val);
          if (A.norm2) nrm += vnorm2(val);
        }
      }
    }
    if (A.norm2) {
      double dn = (double)nrm;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dn += __shfl_down_sync(0xffffffffu, dn, o);
      if (jj == 0) atomicAdd(A.norm2 + rhs, dn);
    }
  }
  if (failed) {
    if (jj == 0) atomicExch(err, 1);
    // drain the copies still in flight (at most one per stage), bounded as well
    for (int s = 0; s < kStages; ++s) mbar_wait_bounded(&bars[s], phase[s]);
  }
}

}  // namespace

template <int OPU, int OPL>
static void launch_tma_variant(const LineArgs<float>& a, int* err, cudaStream_t s) {
  const size_t smem = (size_t)kStages * 18 * a.g.tp * sizeof(Cx<float>) + kStages * sizeof(uint64_t);
  // resident CTAs per SM for this shared-memory size, looked up once (shared by threads)
  static std::mutex mu;
  static std::map<size_t, int> occ;
  int ctas_per_sm = 0, sms = 0, dev = 0;
  WF_CUDA(cudaGetDevice(&dev));
  WF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = occ.find(smem);
    if (it == occ.end()) {
      WF_CUDA(cudaFuncSetAttribute(k_line_tma<OPU, OPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm, k_line_tma<OPU, OPL>, 32, smem));
      if (ctas_per_sm < 1) ctas_per_sm = 1;
      occ[smem] = ctas_per_sm;
    } else {
      ctas_per_sm = it->second;
    }
  }
  WF_CUDA(cudaFuncSetAttribute(k_line_tma<OPU, OPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int lines = a.nrhs * a.g.Nl;
  const int grid = lines < sms * ctas_per_sm ? lines : sms * ctas_per_sm;
  k_line_tma<OPU, OPL><<<grid, 32, smem, s>>>(a, err);
  WF_CUDA(cudaGetLastError());
}

bool tma_supported(const Geom& g) { return g.lpl == 32 && g.lpw == 1 && g.n >= 1 && g.n <= NMAX; }

void launch_line_tma(const LineArgs<float>& a, int kind, int* err, cudaStream_t s) {
  if (!tma_supported(a.g)) throw Error(1, "TMA line kernel needs 32 lanes per line");
  if (kind == LK_SCHUR_B)
    launch_tma_variant<OP_FWD, OP_BWD>(a, err, s);
  else if (kind == LK_SCHUR_C)
    launch_tma_variant<OP_COPY, OP_BWD>(a, err, s);
  else
    throw Error(1, "TMA line kernel: unsupported kind");
}

}  // namespace wf
