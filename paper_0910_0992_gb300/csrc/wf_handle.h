// The handle behind the C ABI and the profiling scope shared by the host-side
// translation units of libwf.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/wf.h"
#include "wf_internal.h"

struct ProfRec {
  int id;
  cudaEvent_t a, b;
};

struct wf_handle {
  wf::Geom g{};
  double xi = 0, kappa_s = 0, kappa_t = 0;
  cudaStream_t stream = 0;
  int device = 0;
  std::string err;
  bool gauge = false;
  bool axial = true;  // solve in the axial frame (U_t = 1 but for P at t = N_t - 1)
  // FP64 line and 4-D dslash operations run in double-float arithmetic while set (the
  // high-precision steps of FP32-iteration solves; see wf_df64.cuh)
  bool df_ops = false;
  bool df_allowed = false;  // double-float steps enabled for this handle
  // while a CG runs: its device flags of active right-hand sides; the Schur operator's kernels
  // skip the others
  const int* op_active = nullptr;
  // gauge, per parity: U_t [Nl][9][tp], spatial [3][Nl][9][tp], Lambda [Nl][9]
  wf::DevBuf ut64[2], us64[2], lamb64[2], lamf64[2];
  wf::DevBuf ut32[2], us32[2], lamb32[2], lamf32[2];
  // axial frame: ut64 holds the rotation g(x) instead of U_t; P per line
  wf::DevBuf pl64[2], pl32[2];
  // clover term of the SW operator (wf_load_gauge_clover): half its chiral blocks per parity,
  // [Nl][2][36][tp]; cleared by wf_load_gauge
  bool clover = false;
  double c_s = 0, c_t = 0;
  wf::DevBuf clov64[2], clov32[2];
  // the same blocks for mu + A and (mu + A)^-1 in the 4-D even-odd layout [L^3][2][36][T/2] per
  // 4-D parity (even T only): the 4-D Schur clover operator
  wf::DevBuf clmu64[2], clmu32[2], clinv64[2], clinv32[2];
  wf::DevBuf tma_err;  // error word of the TMA-fed kernels (bounded waits)
  // index tables of the wide kernels: neighbour lines per parity, traversal order per nrhs
  wf::DevBuf nbr_tab[2];
  std::map<int, std::unique_ptr<wf::DevBuf>> order_tab;  // key: nrhs * 64 + tile rows
  // unit tables of the bulk-fed hop kernels: (first source, line) in traversal order
  std::map<int, std::unique_ptr<wf::DevBuf>> unit_tab;   // key: (nrhs * 64 + tile rows) * 4 + sources per unit
  // autotuned FP32 hop-kernel configuration per nrhs: kernel family (1 one thread per site, 2 n
  // sites per lane, 3 bulk-fed), traversal tile rows, and for the bulk-fed kernels the sources per
  // unit and shared-memory stages
  struct HopTune {
    int variant;
    int by;
    float ms;  // K-b + K-c time of the choice when measured
    int gsrc = 1;
    int ns = 3;
  };
  std::map<int, HopTune> hop_tune;
  int maxiter = 100000;  // CG iteration limit of every solve (wf_set_max_iterations)
  int autotune = -1;  // -1: not decided yet (environment WF_AUTOTUNE=0 keeps the built-in choice)
  int use_tma = -1;    // -1: not decided yet (environment WF_TMA=1 turns the TMA-fed hop kernels on)
  wf::DevBuf iflag;
  std::map<std::string, std::unique_ptr<wf::DevBuf>> ws;  // named work buffers
  // profiling
  bool prof = false;
  std::vector<std::string> prof_names;
  std::map<std::string, int> prof_ids;
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<long long> prof_count;
  std::vector<double> prof_ms;
  long long launches = 0;          // kernels launched by this handle
  double* host_scalars = nullptr;  // pinned

  template <typename T>
  T* buf(const std::string& name, size_t count) {
    auto& b = ws[name];
    if (!b) b.reset(new wf::DevBuf());
    b->ensure(count * sizeof(T), stream);
    return b->as<T>();
  }
  size_t half_int() const { return (size_t)g.Nl * wf::NSPIN_C * g.tp; }  // internal elements, one parity, one rhs
  size_t lex_elems() const { return (size_t)g.L * g.L * g.L * g.T * wf::NSPIN_C; }

  // ---- profiling helpers
  cudaEvent_t take_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    WF_CUDA(cudaEventCreate(&e));
    return e;
  }
  void fold_pending() {
    if (prof_pending.empty()) return;
    WF_CUDA(cudaEventSynchronize(prof_pending.back().b));
    for (auto& r : prof_pending) {
      float ms = 0.f;
      WF_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      prof_ms[r.id] += ms;
      prof_count[r.id] += 1;
      ev_pool.push_back(r.a);
      ev_pool.push_back(r.b);
    }
    prof_pending.clear();
  }
};


namespace wf {

// RAII: CUDA events around one kernel launch when profiling is on
struct Prof {
  wf_handle* h;
  ProfRec rec{};
  bool on;
  Prof(wf_handle* hh, const char* name, int nlaunch = 1) : h(hh), on(hh->prof) {
    h->launches += nlaunch;
    if (!on) return;
    auto it = h->prof_ids.find(name);
    if (it == h->prof_ids.end()) {
      int id = (int)h->prof_names.size();
      h->prof_ids[name] = id;
      h->prof_names.push_back(name);
      h->prof_count.push_back(0);
      h->prof_ms.push_back(0.0);
      rec.id = id;
    } else {
      rec.id = it->second;
    }
    rec.a = h->take_event();
    rec.b = h->take_event();
    WF_CUDA(cudaEventRecord(rec.a, h->stream));
  }
  ~Prof() {
    if (!on) return;
    cudaEventRecord(rec.b, h->stream);
    h->prof_pending.push_back(rec);
    if (h->prof_pending.size() > 4096) {
      try {
        h->fold_pending();
      } catch (...) {
      }
    }
  }
};

// M-hat (dagger: gamma_5 M-hat gamma_5) on internal odd fields x -> out; y (odd) and z (even)
// are work fields of the same size as x.
template <typename R>
void schur_apply(wf_handle* h, const Cx<R>* x, Cx<R>* out, int dagger, int nrhs, Cx<R>* y, Cx<R>* z,
                 double* norm2 = nullptr);

// Whether a caller's array can be used in place on device `dev`: device memory of that GPU or
// managed memory (true), or host memory, pageable or pinned, which the library stages (false).
// Device memory of another GPU is rejected with WF_EINVAL: the kernels would reach it through a
// peer mapping that need not exist.
inline bool device_resident(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) return false;
  if (a.device != dev) throw Error(WF_EINVAL, "array lives on another GPU than the handle's");
  return true;
}

// colour rotation of parity p for imports/exports (axial frame), or null
inline const Cx<double>* frame_rot(const wf_handle* h, int p) {
  return h->axial ? h->ut64[p].as<Cx<double>>() : nullptr;
}

}  // namespace wf
