// Bulk-copy-fed hop kernels K-b and K-c of the Schur operator (FP32, axial frame, 128-slot lines).
//
// The register-fed kernels of wf_wide.cuh keep every hop operand in registers from its load to
// its use. At 72 registers they spill, and they hold about one direction of loads in flight per
// thread, so with twelve sources they wait on memory (long-scoreboard stalls) while neither DRAM,
// L2 nor the issue slots are saturated. Here the operands never pass through registers in flight:
//
// * In the line layout every operand of one hop direction is a contiguous block in HBM: the
//   neighbour line's P_+ and P_- spinor halves (6 x 128 complex each) and the link line in two-row
//   storage (6 x 128 complex). One producer warp brings these blocks into a ring of NS shared-memory
//   stages with cp.async.bulk, completion counted in bytes on a "full" mbarrier per stage; the
//   consumer warps compute a direction from shared memory and release its stage on an "empty"
//   mbarrier. The producer runs NS directions ahead, across unit boundaries, so copies stay in
//   flight while the consumers run the time-line solve of the previous unit.
// * A unit is one line and G sources: the G sources share the stage's link block (G consumer
//   warpgroups of 128 threads, one site per thread), so a link line crosses L2 once per G sources.
// * K-c's post-axpy operand x is one more bulk job per unit (evict-first in L2: read once).
// * The time-line solve is that of wf_wide.cuh (one spin per warp, four sites per thread, a
//   32-lane scan, the wrap closed by K = P Lambda), after a transpose through shared memory.
// * CTAs are persistent: CTA b takes units b, b + grid, ... of the unit table, which lists the
//   (first source, line) pairs in the tiled traversal order of the wide kernels with a line's
//   source groups side by side.
//
// Every wait is bounded (wf_async.cuh). A consumer that gives up makes the whole consumer set
// leave at the next unit boundary (named barrier with an OR reduction, so no warp is left waiting
// at a barrier); the producer then stops issuing and waits, bounded as well, for the copies it
// issued before the CTA's shared memory is released. The host reads the error word and reports
// WF_ETIMEOUT. Tests drive this path by asking the producer to skip one copy, never by a fault.
#include <map>
#include <mutex>

#include "wf_async.cuh"
#include "wf_internal.h"
#include "wf_line.cuh"
#include "wf_wide.cuh"

namespace wf {
namespace pipe {

using namespace async;

constexpr int kTP = 128;                  // slots per line (n = 4 sites per lane group, 32 lanes)
constexpr int kLinkElems = 6 * kTP;       // one link line in two-row storage
constexpr int kHalfElems = 6 * kTP;       // one spin half of one line
constexpr int kSpinElems = 12 * kTP;      // one spinor line
constexpr int kConsBar = 1;               // named barrier of the consumer threads

template <int G>
struct Layout {
  // a stage: the link line, then G spinor lines (P_+ half, P_- half)
  static constexpr int stage_elems = kLinkElems + G * kSpinElems;
  static constexpr size_t stage_bytes = stage_elems * sizeof(Cx<float>);
  // transpose buffer of the time-line solve: [G][12 components][4 sites][32 lanes]
  static constexpr size_t tr_bytes = (size_t)G * 12 * 4 * 32 * sizeof(Cx<float>);
};

template <int G, int NS>
constexpr size_t smem_bytes() {
  return NS * Layout<G>::stage_bytes + Layout<G>::tr_bytes + 2 * NS * sizeof(uint64_t) + 16;
}

// one hop direction d (0: +x, 1: -x, 2: +y, ...) of the site at slot q, from a stage: the same
// arithmetic as wide::hop_site (the projectors' factor 1/2 is applied once, after all six)
__device__ __forceinline__ void hop_dir(Vec3<float> (&h)[4], const Cx<float>* st, const Cx<float>* sp, int q, int d) {
  const int k = d >> 1, dir = d & 1;
  const Vec3<float> u0 = ldvec(sp, kTP, q), u1 = ldvec(sp + 3 * kTP, kTP, q);
  const Vec3<float> d0 = ldvec(sp + 6 * kTP, kTP, q), d1 = ldvec(sp + 9 * kTP, kTP, q);
  const Mat3<float> U = ldlink(st, kTP, q);
  Vec3<float> s0, s1;
  isigma(k, d0, d1, s0, s1);
  Vec3<float> h0, h1;
  if (dir == 0) {
    h0 = vadd(u0, s0);
    h1 = vadd(u1, s1);
  } else {
    h0 = vaxpy(-1.f, s0, u0);
    h1 = vaxpy(-1.f, s1, u1);
  }
  const Vec3<float> w0 = dir == 0 ? matvec(U, h0) : matvec_dag(U, h0);
  const Vec3<float> w1 = dir == 0 ? matvec(U, h1) : matvec_dag(U, h1);
  h[0] = vadd(h[0], w0);
  h[1] = vadd(h[1], w1);
  Vec3<float> r0, r1;
  isigma(k, w0, w1, r0, r1);
  if (dir == 0) {
    h[2] = vaxpy(-1.f, r0, h[2]);
    h[3] = vaxpy(-1.f, r1, h[3]);
  } else {
    h[2] = vadd(h[2], r0);
    h[3] = vadd(h[3], r1);
  }
}

__device__ __forceinline__ bool source_live(const LineArgs<float>& A, int r) {
  return r < A.nrhs && (!A.active || A.active[r]);
}

// a unit is skipped (by producer and consumers alike) when none of its sources is live
template <int G>
__device__ __forceinline__ bool unit_live(const LineArgs<float>& A, const int2* units, int u, int& r0, int& l) {
  const int2 e = units[u];
  r0 = e.x;
  l = e.y;
#pragma unroll
  for (int k = 0; k < G; ++k)
    if (source_live(A, r0 + k)) return true;
  return false;
}

// The producer: lane 0 of the last warp issues every copy of the CTA's units in consumption
// order, NS jobs ahead. Jobs of a unit: the six hop directions, then (K-c) the x operand.
template <int KIND, int G, int NS>
__device__ __forceinline__ void produce(const LineArgs<float>& A, const int2* __restrict__ units, int nunits,
                                        Cx<float>* stage0, uint64_t* full, uint64_t* empty, volatile int* abort_flag,
                                        int* err) {
  constexpr bool KC = KIND == LK_SCHUR_C;
  constexpr int kJobs = KC ? 7 : 6;
  const Geom& g = A.g;
  const int Nl = g.Nl;
  const uint64_t pol_first = policy_evict_first();
  // per-stage bits (bit s for stage s), kept in registers: parity of the next empty phase to wait
  // for, parity of the next full phase, parity of the last full phase issued, stage used at all
  unsigned pe = 0u, pf_next = 0u, pf_last = 0u, used = 0u;
  int job = 0, s = 0;
  bool failed = false;
  for (int u = blockIdx.x; u < nunits && !failed; u += gridDim.x) {
    int r0, l;
    if (!unit_live<G>(A, units, u, r0, l)) continue;
    const int* nbl = A.nbr + (size_t)l * 6;
    for (int jb = 0; jb < kJobs; ++jb, ++job) {
      if (job >= NS) {
        if (!mbar_wait_bounded(&empty[s], (pe >> s) & 1u, abort_flag)) {
          failed = true;
          break;
        }
        pe ^= 1u << s;
      }
      fence_proxy_async();  // the consumers' reads of this stage come before the new copies
      Cx<float>* st = stage0 + (size_t)s * Layout<G>::stage_elems;
      const bool drop = job == A.drop_job && blockIdx.x == 0;  // requested by a test: never lands
      unsigned bytes = 0;
      if (jb < 6) {
        const int k = jb >> 1, ln = nbl[jb];
        const Cx<float>* lk = (jb & 1) == 0 ? A.us_out + ((size_t)k * Nl + l) * kLinkElems
                                            : A.us_nbr + ((size_t)k * Nl + ln) * kLinkElems;
        bytes = kLinkElems * sizeof(Cx<float>);
#pragma unroll
        for (int gg = 0; gg < G; ++gg)
          if (source_live(A, r0 + gg)) bytes += kSpinElems * sizeof(Cx<float>);
        mbar_arrive_expect_tx(&full[s], bytes);
        if (!drop) {
          bulk_g2s(st, lk, kLinkElems * sizeof(Cx<float>), &full[s]);
#pragma unroll
          for (int gg = 0; gg < G; ++gg) {
            if (!source_live(A, r0 + gg)) continue;
            const size_t sb = ((size_t)(r0 + gg) * Nl + ln) * kSpinElems;
            Cx<float>* dst = st + kLinkElems + gg * kSpinElems;
            bulk_g2s(dst, A.src_up + sb, kHalfElems * sizeof(Cx<float>), &full[s]);
            bulk_g2s(dst + kHalfElems, A.src_lo + sb, kHalfElems * sizeof(Cx<float>), &full[s]);
          }
        }
      } else {
#pragma unroll
        for (int gg = 0; gg < G; ++gg)
          if (source_live(A, r0 + gg)) bytes += kSpinElems * sizeof(Cx<float>);
        mbar_arrive_expect_tx(&full[s], bytes);
        if (!drop) {
#pragma unroll
          for (int gg = 0; gg < G; ++gg) {
            if (!source_live(A, r0 + gg)) continue;
            const size_t xb = ((size_t)(r0 + gg) * Nl + l) * kSpinElems;
            bulk_g2s_hint(st + kLinkElems + gg * kSpinElems, A.xpost + xb, kSpinElems * sizeof(Cx<float>), &full[s],
                          pol_first);
          }
        }
      }
      used |= 1u << s;
      pf_last = (pf_last & ~(1u << s)) | (pf_next & (1u << s));
      pf_next ^= 1u << s;
      s = s + 1 == NS ? 0 : s + 1;
    }
  }
  if (failed) {
    atomicExch(err, 1);
    *abort_flag = 1;
  }
  // the last copy issued on every stage must have landed before the CTA's shared memory is freed
#pragma unroll
  for (int k = 0; k < NS; ++k)
    if ((used >> k) & 1u) mbar_wait_bounded(&full[k], (pf_last >> k) & 1u);
}

// K-b: z = C_R^e C_L^e D_s^eo y (T^-dag on the P_+ half, T^-1 on the P_- half);
// K-c: out = x + apost C_L^o D_s^oe z (P_+ half copied, T^-1 on the P_- half), |out|^2.
template <int KIND, int G, int NS>
__global__ void __launch_bounds__(128 * G + 32) k_hop_pipe(const LineArgs<float> A, const int2* __restrict__ units,
                                                           int nunits, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  using Lay = Layout<G>;
  constexpr int kCons = 128 * G;
  constexpr bool KC = KIND == LK_SCHUR_C;
  Cx<float>* stage0 = reinterpret_cast<Cx<float>*>(smem);
  Cx<float>* tr = reinterpret_cast<Cx<float>*>(smem + NS * Lay::stage_bytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * Lay::stage_bytes + Lay::tr_bytes);
  uint64_t* empty = full + NS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NS);
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kCons / 32);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (tid >= kCons) {
    if (tid == kCons) produce<KIND, G, NS>(A, units, nunits, stage0, full, empty, abort_flag, err);
    return;
  }

  const Geom& g = A.g;
  const int Nl = g.Nl;
  const int gi = tid >> 7;                    // this thread's source within the unit
  const int q = tid & 127;                    // its slot of the line
  const int m = q >> 5, j = q & 31;           // warp within the group (= the spin it solves), lane
  const int t = 4 * j + m;                    // the time of slot q
  const int lane = tid & 31;
  Cx<float>* trg = tr + gi * 12 * 4 * 32;     // [12][4][32]
  unsigned pf = 0u;  // bit s: parity of the next full phase of stage s
  int s = 0;
  bool failed = false;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    int r0, l;
    if (!unit_live<G>(A, units, u, r0, l)) continue;
    const int rhs = r0 + gi;
    const bool mine = source_live(A, rhs);
    const bool valid = mine && t < g.T;
    Vec3<float> v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = vzero<float>();
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (!failed && !mbar_wait_bounded(&full[s], (pf >> s) & 1u, abort_flag)) {
        failed = true;
        *abort_flag = 1;  // the others stop waiting too
      }
      pf ^= 1u << s;
      const Cx<float>* st = stage0 + (size_t)s * Lay::stage_elems;
      if (!failed && valid) hop_dir(v, st, st + kLinkElems + gi * kSpinElems, q, d);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      s = s + 1 == NS ? 0 : s + 1;
    }
    int sx = 0;
    if constexpr (KC) {
      sx = s;
      if (!failed && !mbar_wait_bounded(&full[s], (pf >> s) & 1u, abort_flag)) {
        failed = true;
        *abort_flag = 1;
      }
      pf ^= 1u << s;
      s = s + 1 == NS ? 0 : s + 1;
    }
    // every consumer leaves together if one gave up; the barrier also frees the transpose
    // buffer of the previous unit
    if (named_sync_or(kConsBar, kCons, failed)) {
      failed = true;
      break;
    }
    // transposed time-line solve: thread (m, j) hands site t = 4 j + m over and takes back spin m
    // of the four sites of lane group j
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) trg[((3 * sp + c) * 4 + m) * 32 + j] = 0.5f * v[sp].c[c];
    named_sync(kConsBar, kCons);
    const int sp = m, hh = sp >> 1;
    Vec3<float> w[4];
#pragma unroll
    for (int mm = 0; mm < 4; ++mm)
#pragma unroll
      for (int c = 0; c < 3; ++c) w[mm].c[c] = trg[((3 * sp + c) * 4 + mm) * 32 + j];
    const Cx<float>* K_line = A.lamf + (size_t)l * 9;
    if (KIND == LK_SCHUR_B && hh == 0) wide::spin_solve4<float, true>(w, j, g.T, K_line, A.inv_mu, A.bc);
    if (hh == 1) wide::spin_solve4<float, false>(w, j, g.T, K_line, A.inv_mu, A.bc);
    const int dh = A.swap_out ? 1 - hh : hh;
    const int comp0 = dh * 6 + (sp & 1) * 3;
    const size_t base = ((size_t)rhs * Nl + l) * kSpinElems;
    float nrm = 0.f;
    if (mine) {
      const Cx<float>* xs = stage0 + (size_t)sx * Lay::stage_elems + kLinkElems + gi * kSpinElems;
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) {
        const int slot = mm * 32 + j;
        Vec3<float> val = 4 * j + mm < g.T ? w[mm] : vzero<float>();
        if constexpr (KC) val = vaxpy(A.apost, val, ldvec(xs + comp0 * kTP, kTP, slot));
        if (A.stream_out)
          stvec_stream(A.out + base + comp0 * kTP, kTP, slot, val);
        else
          stvec(A.out + base + comp0 * kTP, kTP, slot, val);
        if (A.norm2) nrm += vnorm2(val);
      }
    }
    if constexpr (KC) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sx]);
    }
    if (A.norm2) {
      double dn = (double)nrm;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dn += __shfl_down_sync(0xffffffffu, dn, o);
      if (lane == 0 && mine) atomicAdd(A.norm2 + rhs, dn);
    }
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    *abort_flag = 1;
  }
}

}  // namespace pipe

bool pipe_supported(const Geom& g) { return g.tp == pipe::kTP && g.n == 4 && g.lpl == 32; }

namespace {

template <int KIND, int G, int NS>
void launch_pipe_variant(const LineArgs<float>& a, const int2* units, int nunits, int* err, cudaStream_t s) {
  constexpr size_t smem = pipe::smem_bytes<G, NS>();
  constexpr int threads = 128 * G + 32;
  auto kern = pipe::k_hop_pipe<KIND, G, NS>;
  // per device: shared-memory opt-in and resident CTAs per SM, looked up once
  static std::mutex mu;
  static std::map<int, int> occ;
  int dev = 0, sms = 0, per_sm = 0;
  WF_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = occ.find(dev);
    if (it == occ.end()) {
      WF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
      if (per_sm < 1) throw Error(1, "bulk-fed hop kernel does not fit on an SM");
      occ[dev] = per_sm;
    } else {
      per_sm = it->second;
    }
  }
  WF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = nunits < sms * per_sm ? nunits : sms * per_sm;
  if (grid < 1) return;
  kern<<<grid, threads, smem, s>>>(a, units, nunits, err);
  WF_CUDA(cudaGetLastError());
}

template <int KIND, int G>
void launch_pipe_g(const LineArgs<float>& a, int ns, const int2* units, int nunits, int* err, cudaStream_t s) {
  switch (ns) {
    case 2: launch_pipe_variant<KIND, G, 2>(a, units, nunits, err, s); break;
    case 3: launch_pipe_variant<KIND, G, 3>(a, units, nunits, err, s); break;
    case 4: launch_pipe_variant<KIND, G, 4>(a, units, nunits, err, s); break;
    default: throw Error(1, "bulk-fed hop kernel: unsupported stage count");
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// units: [nunits] (first source, line) pairs; err: device error word (set when a bounded wait expired)
void launch_hop_pipe(const LineArgs<float>& a, int kind, int gsrc, int ns, const int2* units, int nunits, int* err,
                     cudaStream_t s) {
  if (!pipe_supported(a.g)) throw Error(1, "bulk-fed hop kernel: needs 128-slot lines");
  if (!a.nbr || !units || !err) throw Error(1, "bulk-fed hop kernel: neighbour and unit tables and an error word needed");
  if (a.xpre) throw Error(1, "bulk-fed hop kernel: no pre-solve axpy");
  if (!aligned16(a.src_up) || !aligned16(a.src_lo) || !aligned16(a.us_out) || !aligned16(a.us_nbr) ||
      (a.xpost && !aligned16(a.xpost)))
    throw Error(1, "bulk-fed hop kernel: operands must be 16-byte aligned");
  if (kind == LK_SCHUR_C && !a.xpost) throw Error(1, "bulk-fed K-c needs its axpy operand");
  if (kind != LK_SCHUR_B && kind != LK_SCHUR_C) throw Error(1, "bulk-fed hop kernel: K-b or K-c only");
  if (kind == LK_SCHUR_B) {
    if (gsrc == 1) launch_pipe_g<LK_SCHUR_B, 1>(a, ns, units, nunits, err, s);
    else if (gsrc == 2) launch_pipe_g<LK_SCHUR_B, 2>(a, ns, units, nunits, err, s);
    else throw Error(1, "bulk-fed hop kernel: 1 or 2 sources per unit");
  } else {
    if (gsrc == 1) launch_pipe_g<LK_SCHUR_C, 1>(a, ns, units, nunits, err, s);
    else if (gsrc == 2) launch_pipe_g<LK_SCHUR_C, 2>(a, ns, units, nunits, err, s);
    else throw Error(1, "bulk-fed hop kernel: 1 or 2 sources per unit");
  }
}

}  // namespace wf
