// C-ABI of libwf (declared in include/wf.h): handle, gauge ingest, operator applies
// and the CGNR solver for the temporally preconditioned Wilson matrix.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/wf.h"
#include "wf_internal.h"
#include "wf_line.cuh"

using namespace wf;

#include "wf_handle.h"

namespace {


int fail(wf_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

template <typename F>
int guarded(wf_handle* h, F&& f) {
  if (!h) return WF_EINVAL;
  h->err.clear();
  try {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) WF_CUDA(cudaSetDevice(h->device));
    return f();
  } catch (const Error& e) {
    return fail(h, e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(h, WF_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(h, WF_ECUDA, e.what());
  } catch (...) {
    return fail(h, WF_ECUDA, "unknown error");
  }
}

// device view of an input array (staged to the device if it lives on the host)
const Cx<double>* dev_in(wf_handle* h, const double* p, size_t elems, const char* name) {
  if (!p) throw Error(WF_EINVAL, "null array argument");
  if (device_resident(p, h->device)) return reinterpret_cast<const Cx<double>*>(p);
  Cx<double>* d = h->buf<Cx<double>>(name, elems);
  WF_CUDA(cudaMemcpyAsync(d, p, elems * sizeof(Cx<double>), cudaMemcpyHostToDevice, h->stream));
  return d;
}
// device buffer for an output array; finish_out copies it back if the caller's array is host memory
Cx<double>* dev_out(wf_handle* h, double* p, size_t elems, const char* name, bool& staged) {
  if (!p) throw Error(WF_EINVAL, "null array argument");
  staged = !device_resident(p, h->device);
  if (!staged) return reinterpret_cast<Cx<double>*>(p);
  return h->buf<Cx<double>>(name, elems);
}
// a bounded wait in a TMA-fed kernel ran out: report it (the kernels returned without result)
void check_device_error(wf_handle* h) {
  if (!h->tma_err.p) return;
  int e = 0;
  WF_CUDA(cudaMemcpyAsync(&e, h->tma_err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  WF_CUDA(cudaStreamSynchronize(h->stream));
  if (e) {
    WF_CUDA(cudaMemsetAsync(h->tma_err.p, 0, sizeof(int), h->stream));
    throw Error(WF_ETIMEOUT, "a bounded wait for a bulk copy expired in a TMA-fed kernel");
  }
}

void finish_out(wf_handle* h, double* p, const Cx<double>* d, size_t elems, bool staged) {
  if (staged) WF_CUDA(cudaMemcpyAsync(p, d, elems * sizeof(Cx<double>), cudaMemcpyDeviceToHost, h->stream));
  WF_CUDA(cudaStreamSynchronize(h->stream));
  check_device_error(h);
}

// ----------------------------------------------------------------------------
// Gauge views per precision
// ----------------------------------------------------------------------------
template <typename R>
struct Gauge {
  const Cx<R>* ut[2];
  const Cx<R>* pl[2];
  const Cx<R>* us[2];
  const Cx<R>* lamb[2];
  const Cx<R>* lamf[2];
};
template <typename R>
Gauge<R> gauge_of(wf_handle* h);
template <>
Gauge<double> gauge_of<double>(wf_handle* h) {
  Gauge<double> G;
  for (int p = 0; p < 2; ++p) {
    G.ut[p] = h->ut64[p].as<Cx<double>>();
    G.pl[p] = h->pl64[p].as<Cx<double>>();
    G.us[p] = h->us64[p].as<Cx<double>>();
    G.lamb[p] = h->lamb64[p].as<Cx<double>>();
    G.lamf[p] = h->lamf64[p].as<Cx<double>>();
  }
  return G;
}
template <>
Gauge<float> gauge_of<float>(wf_handle* h) {
  Gauge<float> G;
  for (int p = 0; p < 2; ++p) {
    G.ut[p] = h->ut32[p].as<Cx<float>>();
    G.pl[p] = h->pl32[p].as<Cx<float>>();
    G.us[p] = h->us32[p].as<Cx<float>>();
    G.lamb[p] = h->lamb32[p].as<Cx<float>>();
    G.lamf[p] = h->lamf32[p].as<Cx<float>>();
  }
  return G;
}

template <typename R>
LineArgs<R> line_args(wf_handle* h, int parity, int nrhs) {
  Gauge<R> G = gauge_of<R>(h);
  LineArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.g = h->g;
  a.parity = parity;
  a.nrhs = nrhs;
  a.ut = G.ut[parity];
  a.pl = G.pl[parity];
  a.us_out = G.us[parity];
  a.us_nbr = G.us[1 - parity];
  a.lamb = G.lamb[parity];
  a.lamf = G.lamf[parity];
  a.inv_mu = (R)(1.0 / h->g.mu);
  a.bc = (R)h->g.bc;
  a.opu = OP_COPY;
  a.opl = OP_COPY;
  a.drop_job = -1;
  a.df = (sizeof(R) == 8 && h->df_ops) ? 1 : 0;
  return a;
}

// Scope of a solve's double-float FP64 steps: set for FP32-iteration solves, whose reliable
// updates, source preparation and reconstruction then run in double-float; the true residual of
// M stays in FP64 arithmetic.
// Opt-in per handle (environment WF_DF64=1 when the handle is created): measured on GB300
// (16^3 x 128) at 0.9-1.0x the speed of the FP64 kernels, so FP64 arithmetic is the default.
struct DfScope {
  wf_handle* h;
  bool old;
  DfScope(wf_handle* hh, bool on) : h(hh), old(hh->df_ops) { h->df_ops = on && h->df_allowed; }
  ~DfScope() { h->df_ops = old; }
};

// "<base>_f64" / "<base>_f32": buffer and profile names per precision (interned; the map is
// shared by the threads of wf_solve_many)
std::mutex g_pname_mu;
template <typename R>
const char* pname(const char* base);
template <>
const char* pname<double>(const char* base) {
  static std::map<std::string, std::string> m;
  std::lock_guard<std::mutex> lock(g_pname_mu);
  auto& s = m[base];
  if (s.empty()) s = std::string(base) + "_f64";
  return s.c_str();
}
template <>
const char* pname<float>(const char* base) {
  static std::map<std::string, std::string> m;
  std::lock_guard<std::mutex> lock(g_pname_mu);
  auto& s = m[base];
  if (s.empty()) s = std::string(base) + "_f32";
  return s.c_str();
}

// ----------------------------------------------------------------------------
// Operators on internal fields
// ----------------------------------------------------------------------------

// out = C in on one parity: op_up / op_lo per spin half (copy, T^-dag, T^-1)
template <typename R>
void line_load(wf_handle* h, int parity, const Cx<R>* in, Cx<R>* out, int opu, int opl, int nrhs, const char* name) {
  LineArgs<R> a = line_args<R>(h, parity, nrhs);
  a.src_up = in;
  a.src_lo = in + 6 * h->g.tp;
  a.opu = opu;
  a.opl = opl;
  a.src = SRC_LOAD;
  a.out = out;
  Prof P(h, pname<R>(name));
  launch_line<R>(a, LK_GENERIC, h->axial, h->stream);
}

// M-hat (dagger: gamma_5 M-hat gamma_5) on odd internal fields: three fused kernels
//   K-a  y = C_R^o x                        (T^-dag on the upper half only)
//   K-b  z = C_R^e C_L^e D_s^eo y           (hop, then T^-dag upper / T^-1 lower)
//   K-c  out = x - gamma_f^-2 C_L^o D_s^oe z (hop, T^-1 lower, axpy)
// the TMA-fed hop kernels (wf_tma.cu) can serve FP32 in the axial frame with 32 lanes per
// line; they are opt-in (environment WF_TMA=1): on GB300 they measured 1.4-1.8x slower than
// the register-fed line kernel, which keeps twice as many warps resident per SM
template <typename R>
bool use_tma_kernels(wf_handle* h) {
  if (sizeof(R) != 4 || !h->axial || !tma_supported(h->g)) return false;
  if (h->use_tma < 0) {
    const char* e = std::getenv("WF_TMA");
    h->use_tma = (e && e[0] == '1') ? 1 : 0;
  }
  if (h->use_tma && !h->tma_err.p) h->tma_err.ensure(sizeof(int), h->stream);
  return h->use_tma != 0;
}

// Host checks of the kernels' index tables (the kernels index fields through them unchecked):
// every neighbour entry is a line of the other parity whose opposite-direction neighbour is the
// entry's own line; the traversal order visits every (source, line) pair exactly once; the
// bulk-fed kernels' units cover every (source group, line) pair exactly once.
void check_nbr_table(const Geom& g, int p, const std::vector<int>& t) {
  if (t.size() != (size_t)g.Nl * 6) throw Error(WF_ECUDA, "neighbour table: wrong size");
  for (int l = 0; l < g.Nl; ++l)
    for (int d = 0; d < 6; ++d) {
      const int m = t[(size_t)l * 6 + d];
      if (m < 0 || m >= g.Nl) throw Error(WF_ECUDA, "neighbour table: line out of range");
      int back[6];
      neighbour_lines(g, 1 - p, m, back);
      if (back[d ^ 1] != l) throw Error(WF_ECUDA, "neighbour table: not symmetric");
    }
}
void check_order_table(const Geom& g, int nrhs, const std::vector<int2>& t) {
  if (t.size() != (size_t)nrhs * g.Nl) throw Error(WF_ECUDA, "traversal table: wrong size");
  std::vector<char> seen(t.size(), 0);
  for (const int2& e : t) {
    if (e.x < 0 || e.x >= nrhs || e.y < 0 || e.y >= g.Nl) throw Error(WF_ECUDA, "traversal table: entry out of range");
    char& f = seen[(size_t)e.x * g.Nl + e.y];
    if (f) throw Error(WF_ECUDA, "traversal table: pair visited twice");
    f = 1;
  }
}
void check_unit_table(const Geom& g, int nrhs, int gsrc, const std::vector<int2>& t) {
  const int groups = (nrhs + gsrc - 1) / gsrc;
  if (t.size() != (size_t)groups * g.Nl) throw Error(WF_ECUDA, "unit table: wrong size");
  std::vector<char> seen(t.size(), 0);
  for (const int2& e : t) {
    if (e.x < 0 || e.x >= nrhs || e.x % gsrc || e.y < 0 || e.y >= g.Nl) throw Error(WF_ECUDA, "unit table: entry out of range");
    char& f = seen[(size_t)(e.x / gsrc) * g.Nl + e.y];
    if (f) throw Error(WF_ECUDA, "unit table: unit listed twice");
    f = 1;
  }
}
std::vector<int> build_nbr_table(const Geom& g, int p) {
  std::vector<int> t((size_t)g.Nl * 6);
  for (int l = 0; l < g.Nl; ++l) neighbour_lines(g, p, l, &t[(size_t)l * 6]);
  check_nbr_table(g, p, t);
  return t;
}
std::vector<int2> build_order_table(const Geom& g, int nrhs) {
  std::vector<int2> t((size_t)nrhs * g.Nl);
  for (size_t i = 0; i < t.size(); ++i) line_rhs((int)i, nrhs, g, t[i].x, t[i].y);
  check_order_table(g, nrhs, t);
  return t;
}
std::vector<int2> build_unit_table(const Geom& g, int nrhs, int gsrc) {
  const int groups = (nrhs + gsrc - 1) / gsrc;
  std::vector<int2> t((size_t)groups * g.Nl);
  for (int pos = 0; pos < g.Nl; ++pos) {
    int r, l;
    line_rhs(pos, 1, g, r, l);  // with one source the order is the tiled line order itself
    for (int k = 0; k < groups; ++k) t[(size_t)pos * groups + k] = make_int2(k * gsrc, l);
  }
  check_unit_table(g, nrhs, gsrc, t);
  return t;
}

// index tables for the wide kernels (built once per handle and per nrhs, on the handle's stream)
void attach_tables(wf_handle* h, LineArgs<float>& a) {
  const Geom& g = h->g;
  wf::DevBuf& nb = h->nbr_tab[a.parity];
  if (!nb.p) {
    const std::vector<int> t = build_nbr_table(g, a.parity);
    nb.ensure(t.size() * sizeof(int), h->stream);
    WF_CUDA(cudaMemcpyAsync(nb.p, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    WF_CUDA(cudaStreamSynchronize(h->stream));
  }
  auto& ob = h->order_tab[a.nrhs * 64 + a.g.by];
  if (!ob) {
    const std::vector<int2> t = build_order_table(a.g, a.nrhs);
    ob.reset(new wf::DevBuf());
    ob->ensure(t.size() * sizeof(int2), h->stream);
    WF_CUDA(cudaMemcpyAsync(ob->p, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream));
    WF_CUDA(cudaStreamSynchronize(h->stream));
  }
  a.nbr = nb.as<int>();
  a.order = ob->as<int2>();
}

// unit table of the bulk-fed hop kernels: the tiled line order of line_rhs with the sources of a
// line in groups of gsrc side by side, as (first source, line) pairs (built once per handle, nrhs,
// tile rows and group size)
const int2* attach_units(wf_handle* h, const LineArgs<float>& a, int gsrc, int& nunits) {
  const Geom& g = a.g;
  const int groups = (a.nrhs + gsrc - 1) / gsrc;
  nunits = groups * g.Nl;
  auto& ub = h->unit_tab[(a.nrhs * 64 + g.by) * 4 + gsrc];
  if (!ub) {
    const std::vector<int2> t = build_unit_table(g, a.nrhs, gsrc);
    ub.reset(new wf::DevBuf());
    ub->ensure(t.size() * sizeof(int2), h->stream);
    WF_CUDA(cudaMemcpyAsync(ub->p, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream));
    WF_CUDA(cudaStreamSynchronize(h->stream));
  }
  return ub->as<int2>();
}

// one FP32 axial hop launch (K-b or K-c) in the configuration recorded in a.variant (3: the
// bulk-fed kernels with a.pipe_g, a.pipe_ns; else the line kernels)
void launch_hop_config(wf_handle* h, const LineArgs<float>& a0, int kind) {
  LineArgs<float> a = a0;
  attach_tables(h, a);
  if (a.variant == 3) {
    if (!h->tma_err.p) h->tma_err.ensure(sizeof(int), h->stream);
    if (const char* e = std::getenv("WF_TEST_DROP_COPY")) a.drop_job = std::atoi(e);  // fault injection (tests)
    int nunits = 0;
    const int2* units = attach_units(h, a, a.pipe_g, nunits);
    launch_hop_pipe(a, kind, a.pipe_g, a.pipe_ns, units, nunits, h->tma_err.as<int>(), h->stream);
    return;
  }

  launch_line<float>(a, kind, true, h->stream);
}

// Autotuner of the FP32 hop kernels K-b and K-c: the first time a handle applies M-hat to a
// given number of right-hand sides, every candidate -- the register-fed kernels (one thread per
// site or n sites per lane) and, for 128-slot lines, the bulk-fed kernels with 1 or 2 sources per
// unit and 2 to 4 stages, each over traversal tiles of every divisor of L from 2 to 12 rows of y --
// runs K-b and K-c on the call's own buffers, once untimed and three times timed with CUDA
// events; the fastest is kept for the handle. The timed runs write only the work fields K-b and
// K-c own (no norms); the call then computes its result as usual. Environment WF_HOP fixes the
// configuration instead ("wide,<rows>", "lane,<rows>" or "pipe,<sources>,<stages>,<rows>").
static bool autotune_on(wf_handle* h) {
  if (h->autotune < 0) {
    const char* e = std::getenv("WF_AUTOTUNE");
    h->autotune = (e && e[0] == '0') ? 0 : 1;
  }
  return h->autotune != 0;
}

static bool forced_hop(const wf_handle* h, wf_handle::HopTune& t) {
  const char* e = std::getenv("WF_HOP");
  if (!e || !*e) return false;
  int a = 0, b = 0, c = 0;
  if (std::sscanf(e, "pipe,%d,%d,%d", &a, &b, &c) == 3 && pipe_supported(h->g) && (a == 1 || a == 2) && b >= 2 &&
      b <= 4 && c >= 1 && h->g.L % c == 0) {
    t = wf_handle::HopTune{3, c, 0.f, a, b};
    return true;
  }
  if (std::sscanf(e, "wide,%d", &a) == 1 && wide_supported(h->g) && a >= 1 && h->g.L % a == 0) {
    t = wf_handle::HopTune{1, a, 0.f};
    return true;
  }
  if (std::sscanf(e, "lane,%d", &a) == 1 && a >= 1 && h->g.L % a == 0) {
    t = wf_handle::HopTune{2, a, 0.f};
    return true;
  }
  throw Error(WF_EINVAL, std::string("WF_HOP: unknown or unsupported configuration ") + e);
}

static wf_handle::HopTune tune_hops(wf_handle* h, const LineArgs<float>& ab, const LineArgs<float>& ac) {
  wf_handle::HopTune best{0, h->g.by, 0.f};
  if (!h->axial) return best;
  auto it = h->hop_tune.find(ab.nrhs);
  if (it != h->hop_tune.end()) return it->second;
  if (forced_hop(h, best)) {
    h->hop_tune[ab.nrhs] = best;
    return best;
  }
  if (!autotune_on(h)) return best;
  std::vector<int> rows;
  for (int b = 2; b <= 12 && b <= h->g.L; ++b)
    if (h->g.L % b == 0) rows.push_back(b);
  if (rows.empty()) rows.push_back(h->g.by);
  std::vector<wf_handle::HopTune> cands;
  for (int by : rows) {
    if (wide_supported(h->g)) cands.push_back(wf_handle::HopTune{1, by, 0.f});
    cands.push_back(wf_handle::HopTune{2, by, 0.f});
    if (pipe_supported(h->g))
      for (int gs = 1; gs <= 2; ++gs)
        for (int ns = 2; ns <= 4; ++ns)
          if (gs == 1 || ns <= 3) cands.push_back(wf_handle::HopTune{3, by, 0.f, gs, ns});
  }
  cudaEvent_t e0, e1;
  WF_CUDA(cudaEventCreate(&e0));
  WF_CUDA(cudaEventCreate(&e1));
  best.ms = 1e30f;
  for (const auto& cand : cands) {
    LineArgs<float> b = ab, c = ac;
    b.active = c.active = nullptr;
    b.variant = c.variant = cand.variant;
    b.pipe_g = c.pipe_g = cand.gsrc;
    b.pipe_ns = c.pipe_ns = cand.ns;
    b.g.by = c.g.by = cand.by;
    c.norm2 = nullptr;
    float ms = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
      if (rep == 1) WF_CUDA(cudaEventRecord(e0, h->stream));
      launch_hop_config(h, b, LK_SCHUR_B);
      launch_hop_config(h, c, LK_SCHUR_C);
    }
    WF_CUDA(cudaEventRecord(e1, h->stream));
    WF_CUDA(cudaEventSynchronize(e1));
    WF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best.ms) {
      best = cand;
      best.ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->hop_tune[ab.nrhs] = best;
  return best;
}

template <typename R>
void launch_schur_hop(wf_handle* h, const LineArgs<R>& a, int kind, bool tma) {
  if constexpr (sizeof(R) == 4) {
    if (tma) {
      LineArgs<R> b = a;
      if (const char* e = std::getenv("WF_TEST_DROP_COPY")) b.drop_job = std::atoi(e);  // fault injection (tests)
      launch_line_tma(b, kind, h->tma_err.as<int>(), h->stream);
      return;
    }
    if (h->axial) {
      launch_hop_config(h, a, kind);
      return;
    }
  }
  launch_line<R>(a, kind, h->axial, h->stream);
}

}  // namespace

namespace wf {
template <typename R>
void schur_apply(wf_handle* h, const Cx<R>* x, Cx<R>* out, int dagger, int nrhs, Cx<R>* y, Cx<R>* z,
                 double* norm2) {
  const int tp = h->g.tp;
  {
    LineArgs<R> a = line_args<R>(h, 1, nrhs);
    a.active = h->op_active;
    a.src_up = dagger ? x + 6 * tp : x;
    a.src_lo = dagger ? x : x + 6 * tp;
    a.opu = OP_FWD;
    a.opl = OP_SKIP;
    a.out = y;
    Prof P(h, pname<R>("schur_a_tdag"));
    launch_line<R>(a, LK_SCHUR_A, h->axial, h->stream);
  }
  const bool tma = use_tma_kernels<R>(h);
  LineArgs<R> ab = line_args<R>(h, 0, nrhs);
  ab.active = h->op_active;
  ab.src_up = y;
  ab.src_lo = dagger ? x : x + 6 * tp;
  ab.opu = OP_FWD;
  ab.opl = OP_BWD;
  ab.out = z;
  LineArgs<R> ac = line_args<R>(h, 1, nrhs);
  ac.active = h->op_active;
  ac.src_up = z;
  ac.src_lo = z + 6 * tp;
  ac.opu = OP_COPY;
  ac.opl = OP_BWD;
  ac.xpost = x;
  ac.apost = (R)(-1.0 / (h->g.gamma_f * h->g.gamma_f));
  ac.swap_out = dagger;
  ac.stream_out = 1;  // the operator's result is next read by the solver's vector update
  ac.out = out;
  ac.norm2 = norm2;
  if constexpr (sizeof(R) == 4) {
    if (!tma) {
      const wf_handle::HopTune t = tune_hops(h, ab, ac);
      ab.variant = ac.variant = t.variant;
      ab.pipe_g = ac.pipe_g = t.gsrc;
      ab.pipe_ns = ac.pipe_ns = t.ns;
      ab.g.by = ac.g.by = t.by;
    }
  }
  {
    Prof P(h, pname<R>("schur_b_hop_tsolve"));
    launch_schur_hop<R>(h, ab, LK_SCHUR_B, tma);
  }
  {
    if (norm2) WF_CUDA(cudaMemsetAsync(norm2, 0, nrhs * sizeof(double), h->stream));
    Prof P(h, pname<R>("schur_c_hop_tinv_axpy"));
    launch_schur_hop<R>(h, ac, LK_SCHUR_C, tma);
  }
}
template void schur_apply<float>(wf_handle*, const Cx<float>*, Cx<float>*, int, int, Cx<float>*, Cx<float>*,
                                 double*);
template void schur_apply<double>(wf_handle*, const Cx<double>*, Cx<double>*, int, int, Cx<double>*, Cx<double>*,
                                  double*);
}  // namespace wf

namespace {

// out = M in (or x + a M in) on both parities
template <typename R>
void m_apply(wf_handle* h, const Cx<R>* in_e, const Cx<R>* in_o, Cx<R>* out_e, Cx<R>* out_o, const Cx<R>* x_e,
             const Cx<R>* x_o, double a, int nrhs) {
  Gauge<R> G = gauge_of<R>(h);
  for (int p = 0; p < 2; ++p) {
    MArgs<R> m;
    std::memset(&m, 0, sizeof(m));
    m.g = h->g;
    m.parity = p;
    m.nrhs = nrhs;
    m.psi_p = p ? in_o : in_e;
    m.psi_q = p ? in_e : in_o;
    m.ut = G.ut[p];
    m.pl = G.pl[p];
    m.us_out = G.us[p];
    m.us_nbr = G.us[1 - p];
    m.x = p ? x_o : x_e;
    m.a = (R)a;
    m.out = p ? out_o : out_e;
    m.mu = (R)h->g.mu;
    m.inv_gf = (R)(1.0 / h->g.gamma_f);
    m.bc = (R)h->g.bc;
    Prof P(h, pname<R>("apply_M"));
    launch_apply_M<R>(m, h->axial, h->stream);
  }
}

void check_geometry(int L, int T) {
  if (L < 2 || (L & 1)) throw Error(WF_EINVAL, "L must be even and >= 2");
  if (T < 2 || T > 256) throw Error(WF_EINVAL, "T must lie in [2, 256]");
}

// choose sites per lane n and lanes per line lpl (power of two <= 32) with minimal padding; n <= 4
// (the layouts of the fast kernels) whenever T <= 128, else up to 8 (the line kernel's long-line
// variant)
void choose_layout(Geom& g) {
  int best_tp = 1 << 30, best_n = 0, best_lpl = 0;
  for (int n = 1; n <= (g.T <= 32 * NMAX ? NMAX : NMAX_LONG); ++n) {
    int need = (g.T + n - 1) / n;
    int lpl = 1;
    while (lpl < need) lpl <<= 1;
    if (lpl > 32) continue;
    int tp = n * lpl;
    if (tp < best_tp) {
      best_tp = tp;
      best_n = n;
      best_lpl = lpl;
    }
  }
  if (!best_n) throw Error(WF_EINVAL, "T too large for the line layout");
  g.n = best_n;
  g.lpl = best_lpl;
  g.tp = best_tp;
  g.lpw = 32 / best_lpl;
  // traversal tiles of the line kernels: the largest divisor of L up to 8 rows of y
  // (environment WF_TILE_ROWS overrides the bound; L rows is the lexicographic order)
  int max_rows = 8;
  if (const char* e = std::getenv("WF_TILE_ROWS")) {
    const int v = std::atoi(e);
    if (v >= 1) max_rows = v;
  }
  g.by = 1;
  for (int b = 1; b <= g.L && b <= max_rows; ++b)
    if (g.L % b == 0) g.by = b;
}

// the geometry and line layout of an L^3 x T lattice with the given couplings
Geom make_geom(int L, int T, double kappa_s, double kappa_t, int bc) {
  Geom g{};
  g.L = L;
  g.T = T;
  g.Lh = L / 2;
  g.Nl = L * L * L / 2;
  g.mu = 1.0 / (2.0 * kappa_t);
  g.gamma_f = kappa_t / kappa_s;
  g.bc = (double)bc;
  check_geometry(L, T);
  choose_layout(g);
  return g;
}

// ----------------------------------------------------------------------------
// Solver
// ----------------------------------------------------------------------------
struct SolveStats {
  std::vector<int> iters;
  std::vector<double> resid;
};


std::vector<double> read_scalars(wf_handle* h, const double* d, int n) {
  std::vector<double> v(n);
  WF_CUDA(cudaMemcpyAsync(h->host_scalars, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  WF_CUDA(cudaStreamSynchronize(h->stream));
  std::memcpy(v.data(), h->host_scalars, n * sizeof(double));
  check_device_error(h);
  for (double x : v)
    if (!std::isfinite(x)) throw Error(WF_ENAN, "NaN or Inf in a solver norm");
  return v;
}

// A linear operator on internal vectors of one method: y = A x (dagger = 0) or A^dag x
// (dagger = 1) for all right-hand sides; if norm2 is set, |y|^2 per rhs lands there.
template <typename R>
using OpFn = std::function<void(const Cx<R>* x, Cx<R>* y, int dagger, double* norm2)>;

// CGNR, CG on A^dag A y = A^dag b, with operator applies in precision R (R = double: plain
// FP64 CG; R = float: FP32 iterations with FP64 reliable updates of the residual, using A64).
// b and y are FP64 internal vectors of n complex numbers per rhs; stops when |b - A y| <=
// target[k] for every rhs k. Returns the iterations per rhs. reliable = false: no reliable
// updates (A64 is then called only for an initial guess).
template <typename R>
std::vector<int> cgnr(wf_handle* h, const OpFn<R>& A, const OpFn<double>& A64, const Cx<double>* b, Cx<double>* y,
                      int nrhs, size_t n, const std::vector<double>& target, int maxiter, bool x0,
                      size_t ntot = 0, const size_t* offs = nullptr, bool reliable = true) {
  // ragged batches: ntot elements in all, offs the device prefix table of the right-hand sides'
  // first elements (n then the largest length); otherwise nrhs x n
  const size_t nt = ntot ? ntot : n * nrhs;
  cudaStream_t s = h->stream;
  double* sc = h->buf<double>("cg_scalars", 16 * (size_t)nrhs);
  double *gam = sc, *gnew = sc + nrhs, *qq = sc + 2 * nrhs, *rr = sc + 3 * nrhs;
  // device bookkeeping per right-hand side: active, state (0 running, 1 converged, 2 wants a
  // reliable update), iterations; limits: target^2 and the reliable-update threshold^2
  int* ist = h->buf<int>("cg_istate", 4 * (size_t)nrhs);
  int *active = ist, *state = ist + nrhs, *dits = ist + 2 * nrhs;
  int* upd = ist + 3 * nrhs;  // sources whose x update of this iteration is still pending
  double* lim = h->buf<double>("cg_limits", 2 * (size_t)nrhs);
  double* partial = h->buf<double>("cg_partial", 1024 * (size_t)nrhs);
  std::vector<int> act(nrhs, 1), iters(nrhs, 0);
  WF_CUDA(cudaMemcpyAsync(active, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));

  Cx<R>* r = h->buf<Cx<R>>(pname<R>("cg_r"), nt);
  Cx<R>* sv = h->buf<Cx<R>>(pname<R>("cg_s"), nt);
  Cx<R>* p = h->buf<Cx<R>>(pname<R>("cg_p"), nt);
  Cx<R>* q = h->buf<Cx<R>>(pname<R>("cg_q"), nt);
  Cx<R>* xi = h->buf<Cx<R>>(pname<R>("cg_x"), nt);
  Cx<double>* r64 = h->buf<Cx<double>>("cg_r64", nt);
  const bool mixed = sizeof(R) == 4;

  // r64 = b - A y (FP64) or b
  auto true_schur_residual = [&]() {
    const int* keep = h->op_active;
    h->op_active = nullptr;  // every right-hand side's residual
    A64(y, r64, 0, nullptr);
    h->op_active = keep;
    { Prof P(h, "axpby_f64"); launch_axpby<double>(r64, b, nt, 1.0, -1.0, s); }  // r64 = b - A y
  };
  if (x0) {
    true_schur_residual();
  } else {
    WF_CUDA(cudaMemsetAsync(y, 0, nt * sizeof(Cx<double>), s));
    WF_CUDA(cudaMemcpyAsync(r64, b, nt * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, s));
  }
  // working residual in precision R; x increment accumulates in R
  if (mixed) {
    { Prof P(h, "d2f"); launch_d2f(r64, reinterpret_cast<Cx<float>*>(r), nt, s); }
    WF_CUDA(cudaMemsetAsync(xi, 0, nt * sizeof(Cx<R>), s));
  } else {
    WF_CUDA(cudaMemcpyAsync(r, r64, nt * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, s));
  }
  Cx<R>* xacc = mixed ? xi : reinterpret_cast<Cx<R>*>(y);

  { Prof P(h, "norm2_f64", 2); launch_norm2<double>(r64, n, nrhs, partial, rr, s, offs); }
  std::vector<double> rnorm2 = read_scalars(h, rr, nrhs);
  std::vector<double> rmax(nrhs);
  for (int k = 0; k < nrhs; ++k) {
    rmax[k] = std::sqrt(rnorm2[k]);
    if (rnorm2[k] <= target[k] * target[k]) act[k] = 0;
  }
  WF_CUDA(cudaMemcpyAsync(active, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
  auto all_done = [&]() {
    for (int a : act)
      if (a) return false;
    return true;
  };
  if (all_done()) return iters;

  A(r, sv, 1, gam);  // s = A^dag r, |s|^2
  WF_CUDA(cudaMemcpyAsync(p, sv, nt * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, s));

  // reliable-update trigger: the FP32 residual has dropped by this factor since the last
  // FP64 recomputation (environment WF_RELIABLE_DELTA overrides). GB300's FP64 rate makes an
  // FP64 operator apply cost about 15 FP32 ones, so updates are kept few: measured on
  // 24^3 x 128 with 12 sources, 1e-5 gives the iteration counts of 1e-4 .. 1e-2 with fewer
  // FP64 applies.
  double delta = 1e-5;
  if (const char* e = std::getenv("WF_RELIABLE_DELTA")) {
    const double v = std::atof(e);
    if (v > 0.0 && v < 1.0) delta = v;
  }
  // Iterations run in blocks without host synchronisation: convergence and the reliable-update
  // trigger are decided on the device after every x, r update (k_cg_check); the host reads the
  // state once per block, performs reliable updates, and sizes the next block from the observed
  // convergence rate. With a stream of its own and profiling off, one iteration is captured
  // once as a CUDA graph and replayed (environment WF_GRAPH=0: plain launches).
  std::vector<double> tgt2(nrhs), ru2(nrhs);
  std::vector<int> st(nrhs, 0), cnt(nrhs, 0);
  for (int k = 0; k < nrhs; ++k) {
    tgt2[k] = target[k] * target[k];
    ru2[k] = mixed && reliable ? (delta * rmax[k]) * (delta * rmax[k]) : 0.0;
    if (!act[k]) st[k] = 1;
  }
  auto upload_state = [&]() {
    WF_CUDA(cudaMemcpyAsync(active, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
    WF_CUDA(cudaMemcpyAsync(state, st.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
    WF_CUDA(cudaMemcpyAsync(lim, tgt2.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    WF_CUDA(cudaMemcpyAsync(lim + nrhs, ru2.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
  };
  upload_state();
  WF_CUDA(cudaMemsetAsync(dits, 0, nrhs * sizeof(int), s));

  // x += alpha p is deferred from the r update to the p update, which reads p anyway (one pass
  // over the vectors less per iteration); a source that stops at the check still takes it there
  auto iteration = [&]() {
    A(p, q, 0, qq);  // q = A p, |q|^2
    { Prof P(h, pname<R>("cg_xr"), 2); launch_cg_xr<R>(nullptr, r, p, q, n, nrhs, gam, qq, active, partial, rr, s, offs, upd); }
    { Prof P(h, "cg_check"); launch_cg_check(rr, active, state, dits, lim, lim + nrhs, nrhs, s); }
    A(r, sv, 1, gnew);  // s = A^dag r, |s|^2
    { Prof P(h, pname<R>("cg_p")); launch_cg_p<R>(p, sv, n, nrhs, gnew, gam, active, s, offs, xacc, qq, upd); }
    { Prof P(h, "copy_scalar"); launch_copy_scalar(gam, gnew, nrhs, s, active); }
  };

  bool graphs = h->stream != 0 && !h->prof;
  if (const char* e = std::getenv("WF_GRAPH"))
    if (e[0] == '0') graphs = false;
  cudaGraphExec_t gexec = nullptr;
  long long per_iter = 0;
  auto run_block = [&](int nb) {
    for (int i = 0; i < nb; ++i) {
      if (gexec) {
        WF_CUDA(cudaGraphLaunch(gexec, s));
        h->launches += per_iter;
        continue;
      }
      if (graphs && i > 0) {
        // capture one iteration (buffers, tables and tuning already exist after a plain one); the
        // launch counter counts the captured kernels once per replay
        const long long l0 = h->launches;
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        long long captured = 0;
        if (ok) {
          try {
            iteration();
          } catch (...) {
            ok = false;
          }
          captured = h->launches - l0;
          const cudaError_t ee = cudaStreamEndCapture(s, &graph);
          ok = ok && ee == cudaSuccess && graph != nullptr;
          if (ok) ok = cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess;
          if (graph) cudaGraphDestroy(graph);
        }
        (void)cudaGetLastError();  // a failed capture leaves a non-sticky error behind
        h->launches = l0;
        if (!ok) {
          if (gexec) cudaGraphExecDestroy(gexec);
          gexec = nullptr;
          graphs = false;
          iteration();
          continue;
        }
        per_iter = captured;
        WF_CUDA(cudaGraphLaunch(gexec, s));
        h->launches += per_iter;
        continue;
      }
      iteration();
    }
  };

  // the Schur operator's kernels skip right-hand sides that stopped (converged, or waiting for
  // a reliable update) while the blocks run
  struct ActiveScope {
    wf_handle* h;
    ActiveScope(wf_handle* hh, const int* a) : h(hh) { h->op_active = a; }
    ~ActiveScope() { h->op_active = nullptr; }
  } active_scope(h, active);
  std::vector<double> rr_prev(nrhs, 0.0), rrh(nrhs);
  int total = 0, nb = 1;
  while (total < maxiter) {
    nb = std::min(nb, maxiter - total);
    run_block(nb);
    total += nb;
    WF_CUDA(cudaMemcpyAsync(h->host_scalars, rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    int* hist = reinterpret_cast<int*>(h->host_scalars + nrhs);
    WF_CUDA(cudaMemcpyAsync(hist, ist, 3 * nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
    WF_CUDA(cudaStreamSynchronize(s));
    check_device_error(h);
    std::memcpy(rrh.data(), h->host_scalars, nrhs * sizeof(double));
    for (int k = 0; k < nrhs; ++k) {
      if (!std::isfinite(rrh[k])) throw Error(WF_ENAN, "NaN or Inf in a solver norm");
      act[k] = hist[k];
      st[k] = hist[nrhs + k];
      cnt[k] = hist[2 * nrhs + k];
    }
    bool need_ru = false;
    for (int k = 0; k < nrhs; ++k) need_ru = need_ru || st[k] == 2;
    if (need_ru) {
      // reliable update: fold the FP32 increment into y, recompute the residual in FP64. The
      // sources that asked for it stopped right after their x, r update; they now take the rest
      // of that iteration (s = A^dag r, p = s + beta p) with the recomputed residual, the others
      // masked out.
      { Prof P(h, "add_f_to_d"); launch_add_f_to_d(y, reinterpret_cast<const Cx<float>*>(xi), nt, s); }
      WF_CUDA(cudaMemsetAsync(xi, 0, nt * sizeof(Cx<R>), s));
      true_schur_residual();
      { Prof P(h, "norm2_f64", 2); launch_norm2<double>(r64, n, nrhs, partial, rr, s, offs); }
      { Prof P(h, "d2f"); launch_d2f(r64, reinterpret_cast<Cx<float>*>(r), nt, s); }
      std::vector<double> r64n = read_scalars(h, rr, nrhs);
      std::vector<int> resume(nrhs, 0);
      bool any_resume = false;
      for (int k = 0; k < nrhs; ++k) {
        if (st[k] == 1) continue;
        rmax[k] = std::sqrt(r64n[k]);
        ru2[k] = (delta * rmax[k]) * (delta * rmax[k]);
        rrh[k] = r64n[k];
        if (r64n[k] <= tgt2[k]) {
          act[k] = 0;
          st[k] = 1;
        } else if (st[k] == 2) {
          resume[k] = 1;
          any_resume = true;
          st[k] = 0;
          act[k] = 1;
        }
      }
      if (any_resume) {
        WF_CUDA(cudaMemcpyAsync(active, resume.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
        A(r, sv, 1, gnew);
        { Prof P(h, pname<R>("cg_p")); launch_cg_p<R>(p, sv, n, nrhs, gnew, gam, active, s, offs); }
        { Prof P(h, "copy_scalar"); launch_copy_scalar(gam, gnew, nrhs, s, active); }
      }
      upload_state();
    }
    bool done = true;
    for (int a : act) done = done && !a;
    if (done) break;
    // next block: about the iterations the slowest running source still needs at its observed
    // rate (at least 1, at most 16; 2 right after a reliable update)
    // (and no further than the first source's expected reliable-update trigger)
    double need = 1.0, to_ru = 16.0;
    for (int k = 0; k < nrhs; ++k) {
      if (!act[k]) continue;
      const double rho = rr_prev[k] > 0.0 && !need_ru ? std::pow(rrh[k] / rr_prev[k], 1.0 / nb) : 0.0;
      const bool rate = rho > 0.0 && rho < 1.0;
      need = std::max(need, rate ? std::log(tgt2[k] / rrh[k]) / std::log(rho) : 2.0);
      if (mixed && rate && ru2[k] > 0.0 && ru2[k] < rrh[k])
        to_ru = std::min(to_ru, std::log(ru2[k] / rrh[k]) / std::log(rho) + 1.0);
    }
    for (int k = 0; k < nrhs; ++k) rr_prev[k] = rrh[k];
    nb = (int)std::max(1.0, std::min({16.0, std::floor(0.8 * need), std::ceil(to_ru)}));
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  for (int k = 0; k < nrhs; ++k) iters[k] = cnt[k];
  if (mixed) {
    Prof P(h, "add_f_to_d");
    launch_add_f_to_d(y, reinterpret_cast<const Cx<float>*>(xi), nt, s);
  }
  return iters;
}

// M-hat (temporal + 3-D Schur, §II.B) as a CGNR operator on odd internal fields
template <typename R>
OpFn<R> schur_op(wf_handle* h, int nrhs) {
  const size_t nt = h->half_int() * nrhs;
  Cx<R>* ty = h->buf<Cx<R>>(pname<R>("op_ty"), nt);
  Cx<R>* tz = h->buf<Cx<R>>(pname<R>("op_tz"), nt);
  return [=](const Cx<R>* x, Cx<R>* y, int dagger, double* norm2) { schur_apply<R>(h, x, y, dagger, nrhs, ty, tz, norm2); };
}

// M-hat on FP16-stored odd fields, FP32 arithmetic: the kernels of schur_apply<float> (K-a on the
// line kernel, K-b / K-c on the one-thread-per-site kernels in the tuned traversal) with FP16
// loads and stores. Element offsets of FP16 fields are taken in Cx16 units before the pointer
// is carried as Cx<float>*.
void schur_apply_h16(wf_handle* h, const Cx16* x, Cx16* out, int dagger, int nrhs, Cx16* y, Cx16* z, double* norm2) {
  const int tp = h->g.tp;
  auto F = [](const Cx16* q) { return reinterpret_cast<const Cx<float>*>(q); };
  auto W = [](Cx16* q) { return reinterpret_cast<Cx<float>*>(q); };
  {
    LineArgs<float> a = line_args<float>(h, 1, nrhs);
    a.h16 = 1;
    a.active = h->op_active;
    a.src_up = F(dagger ? x + 6 * tp : x);
    a.src_lo = F(dagger ? x : x + 6 * tp);
    a.opu = OP_FWD;
    a.opl = OP_SKIP;
    a.out = W(y);
    Prof P(h, "schur_a_tdag_h16");
    launch_line<float>(a, LK_SCHUR_A, h->axial, h->stream);
  }
  auto it = h->hop_tune.find(nrhs);
  const int by = it != h->hop_tune.end() ? it->second.by : h->g.by;
  LineArgs<float> ab = line_args<float>(h, 0, nrhs);
  ab.h16 = 1;
  ab.active = h->op_active;
  ab.src_up = F(y);
  ab.src_lo = F(dagger ? x : x + 6 * tp);
  ab.opu = OP_FWD;
  ab.opl = OP_BWD;
  ab.out = W(z);
  ab.variant = 1;
  ab.g.by = by;
  LineArgs<float> ac = line_args<float>(h, 1, nrhs);
  ac.h16 = 1;
  ac.active = h->op_active;
  ac.src_up = F(z);
  ac.src_lo = F(z + 6 * tp);
  ac.opu = OP_COPY;
  ac.opl = OP_BWD;
  ac.xpost = F(x);
  ac.apost = (float)(-1.0 / (h->g.gamma_f * h->g.gamma_f));
  ac.swap_out = dagger;
  ac.stream_out = 1;
  ac.out = W(out);
  ac.norm2 = norm2;
  ac.variant = 1;
  ac.g.by = by;
  {
    Prof P(h, "schur_b_hop_tsolve_h16");
    launch_hop_config(h, ab, LK_SCHUR_B);
  }
  {
    if (norm2) WF_CUDA(cudaMemsetAsync(norm2, 0, nrhs * sizeof(double), h->stream));
    Prof P(h, "schur_c_hop_tinv_axpy_h16");
    launch_hop_config(h, ac, LK_SCHUR_C);
  }
}

// CGNR with FP16-stored vectors (FP32 arithmetic) and reliable updates on two levels, for
// the FP16MIX precision. The vectors r, s, p, q of each right-hand side are stored divided by
// a scale sigma (the RMS of its residual at the last reliable update), so they stay O(1) in
// FP16. The iterate is accumulated in FP32 (true units) as the increment xi since the last FP64
// update. A right-hand side asks for a reliable update when its iterated residual fell by
// delta16 since the last one, or reached its target (then the recomputed residual decides):
//   * FP32 update: r = r64 - A32 xi, the FP32 residual of the increment against the FP64
//     residual r64 of the last FP64 update (accurate to ~1e-7 of |r64|, as xi is small);
//   * FP64 update, when a requesting residual fell below delta64 |r64|: y += xi, xi = 0,
//     r64 = b - A64 y.
// Every update refreshes r for all right-hand sides and rescales r, p and gamma by the new
// sigma; the requesting right-hand sides then finish their iteration (s = A^dag r, p = s + beta
// p). Iterations run in blocks with device-side checks (k_cg_check) as in cgnr; no CUDA graph.
std::vector<int> cgnr_h16(wf_handle* h, int nrhs, size_t n, const Cx<double>* b, Cx<double>* y,
                          const std::vector<double>& target, int maxiter, bool x0, bool fp64_updates = true) {
  const size_t nt = n * nrhs;
  cudaStream_t s = h->stream;
  const OpFn<float> A32 = schur_op<float>(h, nrhs);
  const OpFn<double> A64 = schur_op<double>(h, nrhs);
  Cx16* r = h->buf<Cx16>("h16_r", nt);
  Cx16* sv = h->buf<Cx16>("h16_s", nt);
  Cx16* p = h->buf<Cx16>("h16_p", nt);
  Cx16* q = h->buf<Cx16>("h16_q", nt);
  Cx16* ty = h->buf<Cx16>("h16_ty", nt);
  Cx16* tz = h->buf<Cx16>("h16_tz", nt);
  Cx<float>* xi = h->buf<Cx<float>>("h16_xi", nt);
  Cx<float>* t32 = h->buf<Cx<float>>("h16_t32", nt);
  Cx<float>* r32 = h->buf<Cx<float>>("h16_r32", nt);
  Cx<double>* r64 = h->buf<Cx<double>>("cg_r64", nt);
  double* sc = h->buf<double>("h16_scalars", 8 * (size_t)nrhs);
  double *gam = sc, *gnew = sc + nrhs, *qq = sc + 2 * nrhs, *rr = sc + 3 * nrhs, *sig = sc + 4 * nrhs,
         *fac = sc + 5 * nrhs;
  int* ist = h->buf<int>("cg_istate", 3 * (size_t)nrhs);
  int *active = ist, *state = ist + nrhs, *dits = ist + 2 * nrhs;
  double* lim = h->buf<double>("cg_limits", 2 * (size_t)nrhs);
  double* partial = h->buf<double>("cg_partial", 1024 * (size_t)nrhs);
  auto A16 = [&](const Cx16* in, Cx16* out, int dagger, double* norm2) {
    schur_apply_h16(h, in, out, dagger, nrhs, ty, tz, norm2);
  };
  double d16 = 1e-2, d64 = 1e-5;
  if (const char* e = std::getenv("WF_RELIABLE_DELTA16")) {
    const double v = std::atof(e);
    if (v > 0.0 && v < 1.0) d16 = v;
  }
  if (const char* e = std::getenv("WF_RELIABLE_DELTA")) {
    const double v = std::atof(e);
    if (v > 0.0 && v < 1.0) d64 = v;
  }
  std::vector<int> act(nrhs, 1), st(nrhs, 0), cnt(nrhs, 0), iters(nrhs, 0);
  std::vector<double> sigma(nrhs, 1.0), rmax(nrhs), rlast(nrhs), tgt2(nrhs), ru2(nrhs), f(nrhs, 1.0);
  auto upload = [&](double* dst, const std::vector<double>& v) {
    WF_CUDA(cudaMemcpyAsync(dst, v.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
  };
  auto upload_state = [&]() {
    for (int k = 0; k < nrhs; ++k) {
      tgt2[k] = (target[k] / sigma[k]) * (target[k] / sigma[k]);
      ru2[k] = (d16 * rlast[k] / sigma[k]) * (d16 * rlast[k] / sigma[k]);
    }
    WF_CUDA(cudaMemcpyAsync(active, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
    WF_CUDA(cudaMemcpyAsync(state, st.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
    upload(lim, tgt2);
    upload(lim + nrhs, ru2);
    upload(sig, sigma);
  };
  // new scales from the residual norms r2 (true units); rescale p and gamma of every rhs by
  // old / new sigma and store r (true units, in src) scaled into FP16
  auto rescale = [&](const std::vector<double>& r2, auto* src, bool with_p) {
    for (int k = 0; k < nrhs; ++k) {
      const double sn = r2[k] > 0.0 ? std::sqrt(r2[k] / (double)n) : sigma[k];
      f[k] = sigma[k] / sn;
      sigma[k] = sn;
    }
    std::vector<double> inv(nrhs), f2(nrhs);
    for (int k = 0; k < nrhs; ++k) {
      inv[k] = 1.0 / sigma[k];
      f2[k] = f[k] * f[k];
    }
    upload(fac, inv);
    { Prof P(h, "h16_scale_r"); launch_scale_to_h16(r, src, n, nrhs, fac, s); }
    if (with_p) {
      upload(fac, f);
      { Prof P(h, "h16_scale_p"); launch_scale_to_h16<Cx16>(p, p, n, nrhs, fac, s); }
      std::vector<double> g = read_scalars(h, gam, nrhs);
      for (int k = 0; k < nrhs; ++k) g[k] *= f2[k];
      upload(gam, g);
    }
  };

  // r64 = b - A y, or b
  if (x0) {
    const int* keep = h->op_active;
    h->op_active = nullptr;
    A64(y, r64, 0, nullptr);
    h->op_active = keep;
    { Prof P(h, "axpby_f64"); launch_axpby<double>(r64, b, nt, 1.0, -1.0, s); }
  } else {
    WF_CUDA(cudaMemsetAsync(y, 0, nt * sizeof(Cx<double>), s));
    WF_CUDA(cudaMemcpyAsync(r64, b, nt * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, s));
  }
  WF_CUDA(cudaMemsetAsync(xi, 0, nt * sizeof(Cx<float>), s));
  { Prof P(h, "norm2_f64", 2); launch_norm2<double>(r64, n, nrhs, partial, rr, s); }
  std::vector<double> r2 = read_scalars(h, rr, nrhs);
  for (int k = 0; k < nrhs; ++k) {
    rmax[k] = rlast[k] = std::sqrt(r2[k]);
    if (r2[k] <= target[k] * target[k]) {
      act[k] = 0;
      st[k] = 1;
    }
  }
  bool done = true;
  for (int a : act) done = done && !a;
  if (done) return iters;
  rescale(r2, r64, false);
  upload_state();
  struct ActiveScope {
    wf_handle* h;
    ActiveScope(wf_handle* hh, const int* a) : h(hh) { h->op_active = a; }
    ~ActiveScope() { h->op_active = nullptr; }
  } active_scope(h, active);
  A16(r, sv, 1, gam);  // s = A^dag r, gamma = |s|^2
  WF_CUDA(cudaMemcpyAsync(p, sv, nt * sizeof(Cx16), cudaMemcpyDeviceToDevice, s));
  WF_CUDA(cudaMemsetAsync(dits, 0, nrhs * sizeof(int), s));

  auto iteration = [&]() {
    A16(p, q, 0, qq);  // q = A p, |q|^2
    { Prof P(h, "cg_xr_h16", 2); launch_cg_xr_h16(xi, r, p, q, n, nrhs, gam, qq, sig, active, partial, rr, s); }
    { Prof P(h, "cg_check"); launch_cg_check(rr, active, state, dits, lim, lim + nrhs, nrhs, s); }
    A16(r, sv, 1, gnew);  // s = A^dag r, |s|^2
    { Prof P(h, "cg_p_h16"); launch_cg_p_h16(p, sv, n, nrhs, gnew, gam, active, s); }
    { Prof P(h, "copy_scalar"); launch_copy_scalar(gam, gnew, nrhs, s, active); }
  };

  std::vector<double> rrh(nrhs), rr_prev(nrhs, 0.0);
  int total = 0, nb = 1;
  while (total < maxiter) {
    nb = std::min(nb, maxiter - total);
    for (int i = 0; i < nb; ++i) iteration();
    total += nb;
    WF_CUDA(cudaMemcpyAsync(h->host_scalars, rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    int* hist = reinterpret_cast<int*>(h->host_scalars + nrhs);
    WF_CUDA(cudaMemcpyAsync(hist, ist, 3 * nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
    WF_CUDA(cudaStreamSynchronize(s));
    check_device_error(h);
    std::memcpy(rrh.data(), h->host_scalars, nrhs * sizeof(double));
    bool need = false, need64 = false;
    for (int k = 0; k < nrhs; ++k) {
      if (!std::isfinite(rrh[k])) throw Error(WF_ENAN, "NaN or Inf in a solver norm");
      act[k] = hist[k];
      const int sk = hist[nrhs + k];
      cnt[k] = hist[2 * nrhs + k];
      if (st[k] != 1 && sk != 0) {  // asks for an update (its residual fell by delta16 or met its target)
        need = true;
        st[k] = 2;
        if (fp64_updates && sigma[k] * std::sqrt(rrh[k]) < d64 * rmax[k]) need64 = true;
      }
    }
    if (need) {
      std::vector<double> nr2;
      if (need64) {
        { Prof P(h, "add_f_to_d"); launch_add_f_to_d(y, xi, nt, s); }
        WF_CUDA(cudaMemsetAsync(xi, 0, nt * sizeof(Cx<float>), s));
        const int* keep = h->op_active;
        h->op_active = nullptr;
        A64(y, r64, 0, nullptr);
        h->op_active = keep;
        { Prof P(h, "axpby_f64"); launch_axpby<double>(r64, b, nt, 1.0, -1.0, s); }  // r64 = b - A y
        { Prof P(h, "norm2_f64", 2); launch_norm2<double>(r64, n, nrhs, partial, rr, s); }
        nr2 = read_scalars(h, rr, nrhs);
        rescale(nr2, r64, true);
        for (int k = 0; k < nrhs; ++k) rmax[k] = rlast[k] = std::sqrt(nr2[k]);
      } else {
        const int* keep = h->op_active;
        h->op_active = nullptr;
        A32(xi, t32, 0, nullptr);  // A32 xi
        h->op_active = keep;
        { Prof P(h, "h16_sub"); launch_sub_d_f(r32, r64, t32, nt, s); }  // r = r64 - A32 xi
        { Prof P(h, "norm2_f32", 2); launch_norm2<float>(r32, n, nrhs, partial, rr, s); }
        nr2 = read_scalars(h, rr, nrhs);
        rescale(nr2, r32, true);
        for (int k = 0; k < nrhs; ++k) rlast[k] = std::sqrt(nr2[k]);
      }
      std::vector<int> resume(nrhs, 0);
      bool any_resume = false;
      for (int k = 0; k < nrhs; ++k) {
        if (st[k] == 1) continue;
        if (nr2[k] <= target[k] * target[k]) {
          act[k] = 0;
          st[k] = 1;
        } else if (st[k] == 2) {
          resume[k] = 1;
          any_resume = true;
          st[k] = 0;
          act[k] = 1;
        }
      }
      if (any_resume) {
        WF_CUDA(cudaMemcpyAsync(active, resume.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
        A16(r, sv, 1, gnew);
        { Prof P(h, "cg_p_h16"); launch_cg_p_h16(p, sv, n, nrhs, gnew, gam, active, s); }
        { Prof P(h, "copy_scalar"); launch_copy_scalar(gam, gnew, nrhs, s, active); }
      }
      upload_state();
    }
    done = true;
    for (int a : act) done = done && !a;
    if (done) break;
    // next block: most of the iterations until the first running source's expected next update
    // (at least 1, at most 16; 2 right after an update), so that few launches find every source
    // stopped
    double need_it = 16.0;
    for (int k = 0; k < nrhs; ++k) {
      if (!act[k]) continue;
      const double rho = rr_prev[k] > 0.0 && !need ? std::pow(rrh[k] / rr_prev[k], 1.0 / nb) : 0.0;
      if (rho > 0.0 && rho < 1.0)
        need_it = std::min(need_it, std::log(std::max(ru2[k], tgt2[k]) / rrh[k]) / std::log(rho));
    }
    for (int k = 0; k < nrhs; ++k) rr_prev[k] = rrh[k];
    nb = need ? 2 : (int)std::max(1.0, std::min(16.0, std::floor(0.8 * need_it)));
  }
  for (int k = 0; k < nrhs; ++k) iters[k] = cnt[k];
  { Prof P(h, "add_f_to_d"); launch_add_f_to_d(y, xi, nt, s); }
  return iters;
}

// Temporal + 3-D Schur solve (§II.B): prepare with S_L, CGNR on M-hat, reconstruct with S_R,
// verify with the FP64 true residual of M.
void solve_temporal_schur_dc(int nl, wf_handle* const* hs, const std::vector<const Cx<double>*>& eta_lex,
                             const std::vector<Cx<double>*>& x_lex, const int* nrhs, double tol, bool x0,
                             std::vector<std::vector<int>>& iters, std::vector<std::vector<double>>& rel,
                             std::vector<int>& status, bool h16 = false);

// FP32 temporal + Schur solves take defect correction (solve_temporal_schur_dc) unless the
// environment sets WF_DC=0, which selects FP32 iterations with FP64 reliable updates
bool use_defect_correction() {
  const char* e = std::getenv("WF_DC");
  return !(e && e[0] == '0');
}

int solve_temporal_schur(wf_handle* h, const Cx<double>* eta_lex, Cx<double>* x_lex, int nrhs, double tol,
                         int precision, bool x0, int* iters_out, double* resid_out) {
  if ((precision == WF_FP32 || precision == WF_FP16MIX) && use_defect_correction()) {
    std::vector<std::vector<int>> it(1);
    std::vector<std::vector<double>> res(1);
    std::vector<int> st(1);
    wf_handle* const hs[1] = {h};
    solve_temporal_schur_dc(1, hs, {eta_lex}, {x_lex}, &nrhs, tol, x0, it, res, st, precision == WF_FP16MIX);
    for (int k = 0; k < nrhs; ++k) {
      if (iters_out) iters_out[k] = it[0][k];
      if (resid_out) resid_out[k] = res[0][k];
    }
    return st[0];
  }
  const size_t n = h->half_int();
  const size_t nt = n * nrhs;
  cudaStream_t s = h->stream;
  DfScope dfs(h, precision == WF_FP32);
  const double igf = 1.0 / h->g.gamma_f;
  Cx<double>* eta_e = h->buf<Cx<double>>("sv_eta_e", nt);
  Cx<double>* eta_o = h->buf<Cx<double>>("sv_eta_o", nt);
  Cx<double>* a_e = h->buf<Cx<double>>("sv_a_e", nt);
  Cx<double>* b_o = h->buf<Cx<double>>("sv_b_o", nt);
  Cx<double>* y_o = h->buf<Cx<double>>("sv_y_o", nt);
  Cx<double>* psi_e = h->buf<Cx<double>>("sv_psi_e", nt);
  Cx<double>* psi_o = h->buf<Cx<double>>("sv_psi_o", nt);
  Cx<double>* r_e = h->buf<Cx<double>>("sv_r_e", nt);
  Cx<double>* r_o = h->buf<Cx<double>>("sv_r_o", nt);
  double* sc = h->buf<double>("sv_scalars", 4 * (size_t)nrhs);
  double* partial = h->buf<double>("cg_partial", 1024 * (size_t)nrhs);

  { Prof P(h, "import_spinor_f64"); launch_import_spinor<double>(h->g, eta_lex, eta_e, eta_o, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), s); }
  // source preparation (S_L): a_e = C_R^e C_L^e eta_e ; b_o = C_L^o [eta_o + gamma_f^-1 D_s^oe a_e]
  line_load<double>(h, 0, eta_e, a_e, OP_FWD, OP_BWD, nrhs, "prep_tsolve");
  {
    LineArgs<double> a = line_args<double>(h, 1, nrhs);
    a.src_up = a_e;
    a.src_lo = a_e + 6 * h->g.tp;
    a.xpre = eta_o;
    a.apre = igf;
    a.opu = OP_COPY;
    a.opl = OP_BWD;
    a.src = SRC_HOP;
    a.out = b_o;
    Prof P(h, "prep_hop_f64");
    launch_line<double>(a, LK_GENERIC, h->axial, s);
  }
  // |eta|^2 per rhs
  { Prof P(h, "norm2_f64", 4); launch_norm2<double>(eta_e, n, nrhs, partial, sc, s); launch_norm2<double>(eta_o, n, nrhs, partial, sc + nrhs, s); }
  std::vector<double> e2 = read_scalars(h, sc, 2 * nrhs);
  std::vector<double> eta2(nrhs), target(nrhs);
  for (int k = 0; k < nrhs; ++k) {
    eta2[k] = e2[k] + e2[nrhs + k];
    // |eta - M psi| = |C_L^o^-1 r_o| <= (mu + 1) |r_o|
    target[k] = tol * std::sqrt(eta2[k]) / (h->g.mu + 1.0);
  }
  bool have_x0 = x0;
  if (x0) {
    // initial guess: y_o = (C_R^o)^-1 psi_o; use only the odd part of the guess
    Cx<double>* g_e = r_e;
    { Prof P(h, "import_spinor_f64"); launch_import_spinor<double>(h->g, x_lex, g_e, psi_o, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), s); }
    // (C_R^o)^-1 = P_- + P_+ T^dag is not needed exactly: start from y_o = psi_o
    WF_CUDA(cudaMemcpyAsync(y_o, psi_o, nt * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, s));
  }
  std::vector<int> iters(nrhs, 0);
  std::vector<double> rel(nrhs, 0.0);
  const int maxiter = h->maxiter;
  int status = WF_OK;
  for (int pass = 0; pass < 6; ++pass) {
    std::vector<int> it = precision == WF_FP16MIX
                              ? cgnr_h16(h, nrhs, n, b_o, y_o, target, maxiter, have_x0)
                          : precision == WF_FP32
                              ? cgnr<float>(h, schur_op<float>(h, nrhs), schur_op<double>(h, nrhs), b_o, y_o, nrhs, n,
                                            target, maxiter, have_x0)
                              : cgnr<double>(h, schur_op<double>(h, nrhs), schur_op<double>(h, nrhs), b_o, y_o, nrhs,
                                             n, target, maxiter, have_x0);
    for (int k = 0; k < nrhs; ++k) iters[k] += it[k];
    have_x0 = true;
    // reconstruction (S_R): psi_o = C_R^o y_o ; psi_e = C_R^e C_L^e [eta_e + gamma_f^-1 D_s^eo psi_o]
    line_load<double>(h, 1, y_o, psi_o, OP_FWD, OP_COPY, nrhs, "recon_tsolve");
    {
      LineArgs<double> a = line_args<double>(h, 0, nrhs);
      a.src_up = psi_o;
      a.src_lo = psi_o + 6 * h->g.tp;
      a.xpre = eta_e;
      a.apre = igf;
      a.opu = OP_FWD;
      a.opl = OP_BWD;
      a.src = SRC_HOP;
      a.out = psi_e;
      Prof P(h, "recon_hop_f64");
      launch_line<double>(a, LK_GENERIC, h->axial, s);
    }
    // true residual r = eta - M psi in FP64
    m_apply<double>(h, psi_e, psi_o, r_e, r_o, eta_e, eta_o, -1.0, nrhs);
    { Prof P(h, "norm2_f64", 4); launch_norm2<double>(r_e, n, nrhs, partial, sc, s); launch_norm2<double>(r_o, n, nrhs, partial, sc + nrhs, s); }
    std::vector<double> r2 = read_scalars(h, sc, 2 * nrhs);
    bool ok = true;
    for (int k = 0; k < nrhs; ++k) {
      rel[k] = std::sqrt((r2[k] + r2[nrhs + k]) / (eta2[k] > 0 ? eta2[k] : 1.0));
      if (rel[k] > tol) {
        ok = false;
        target[k] *= 0.5 * tol / rel[k];
      }
      if (iters[k] >= maxiter) status = WF_ENOCONV;
    }
    if (ok || status == WF_ENOCONV) break;
    if (pass == 5) status = WF_ENOCONV;
  }
  { Prof P(h, "export_spinor_f64"); launch_export_spinor<double>(h->g, psi_e, psi_o, x_lex, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), s); }
  for (int k = 0; k < nrhs; ++k) {
    if (iters_out) iters_out[k] = iters[k];
    if (resid_out) resid_out[k] = rel[k];
  }
  return status;
}

// ----------------------------------------------------------------------------
// Ragged batches: one temporal + Schur solve over several lattices (wf_solve_many)
// ----------------------------------------------------------------------------

// One lattice of a joint solve: its handle, sources, field length and place in the joint vectors
struct JointPart {
  wf_handle* h;
  int nrhs;
  size_t n;    // complex numbers per source (odd internal field)
  size_t off;  // first element of its sources in the joint vectors
  int r0;      // its first source in the joint numbering
};

// Events ordering the joint stream (hs[0]'s) and the lattices' own streams: fan_out makes every
// lattice's stream wait for the joint stream's work so far, fan_in the joint stream for theirs
struct JointSync {
  std::vector<cudaEvent_t> ev;
  explicit JointSync(size_t n) : ev(n + 1, nullptr) {
    for (auto& e : ev) WF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  ~JointSync() {
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  }
  void fan_out(const std::vector<JointPart>& parts) const {
    cudaStream_t s0 = parts[0].h->stream;
    WF_CUDA(cudaEventRecord(ev[0], s0));
    for (size_t j = 1; j < parts.size(); ++j) WF_CUDA(cudaStreamWaitEvent(parts[j].h->stream, ev[0], 0));
  }
  void fan_in(const std::vector<JointPart>& parts) const {
    cudaStream_t s0 = parts[0].h->stream;
    for (size_t j = 1; j < parts.size(); ++j) {
      WF_CUDA(cudaEventRecord(ev[j], parts[j].h->stream));
      WF_CUDA(cudaStreamWaitEvent(s0, ev[j], 0));
    }
  }
};

// M-hat of every lattice in FP32, with x, y, the norms and the solver's active flags in the joint
// numbering, on the joint stream. K-a runs as one launch over all lattices' sources (per
// kMaxLattices lattices). K-b and K-c take each lattice's autotuned configuration (the tuner runs
// here, on scratch fields, for a handle that has none for its number of sources): the lattices
// whose choice is the one-thread-per-site kernels share one launch per kernel (two: 128-slot lines
// and the others), so do those on n sites per lane, and the bulk-fed ones launch their own.
// Tables are attached here, before the solver captures an iteration.
OpFn<float> joint_schur_op(const std::vector<JointPart>& parts, Cx<float>* ty, Cx<float>* tz, Cx<float>* tw,
                           int nr) {
  wf_handle* h0 = parts[0].h;
  struct Own {
    LineArgs<float> b, c;
    wf_handle::HopTune t;
    const int2* units;
    int nunits;
    int* err;
  };
  std::vector<LineArgs<float>> A, B, C;  // K-a of all; K-b, K-c of the lattices on the shared launches
  std::vector<LineArgs<float>> B2, C2;   // K-b, K-c of the lattices on n sites per lane
  std::vector<int> joined, joined2;      // lattice of each B/C and B2/C2 entry
  std::vector<std::pair<int, Own>> own;  // lattices with a launch of their own (bulk-fed kernels)
  for (int j = 0; j < (int)parts.size(); ++j) {
    const JointPart& q = parts[j];
    wf_handle* h = q.h;
    const int tp = h->g.tp;
    LineArgs<float> a = line_args<float>(h, 1, q.nrhs);
    a.opu = OP_FWD;
    a.opl = OP_SKIP;
    a.out = ty + q.off;
    LineArgs<float> b = line_args<float>(h, 0, q.nrhs);
    b.src_up = ty + q.off;
    b.opu = OP_FWD;
    b.opl = OP_BWD;
    b.out = tz + q.off;
    LineArgs<float> c = line_args<float>(h, 1, q.nrhs);
    c.src_up = tz + q.off;
    c.src_lo = tz + q.off + 6 * tp;
    c.opu = OP_COPY;
    c.opl = OP_BWD;
    c.apost = (float)(-1.0 / (h->g.gamma_f * h->g.gamma_f));
    c.stream_out = 1;
    // the tuner times K-b and K-c on scratch fields of this lattice's size
    LineArgs<float> bt = b, ct = c;
    bt.src_lo = ty + q.off;
    ct.xpost = ty + q.off;
    ct.out = tw + q.off;
    const wf_handle::HopTune t = tune_hops(h, bt, ct);
    b.variant = c.variant = t.variant;
    b.pipe_g = c.pipe_g = t.gsrc;
    b.pipe_ns = c.pipe_ns = t.ns;
    b.g.by = c.g.by = t.by;
    attach_tables(h, b);
    attach_tables(h, c);
    A.push_back(a);
    if (t.variant <= 1) {
      B.push_back(b);
      C.push_back(c);
      joined.push_back(j);
    } else if (t.variant == 2) {
      B2.push_back(b);
      C2.push_back(c);
      joined2.push_back(j);
    } else {
      Own o{b, c, t, nullptr, 0, nullptr};
      if (t.variant == 3) {
        o.units = attach_units(h, b, t.gsrc, o.nunits);
        if (!h->tma_err.p) h->tma_err.ensure(sizeof(int), h->stream);
        o.err = h->tma_err.as<int>();
      }
      own.emplace_back(j, o);
    }
  }
  const int nl = (int)parts.size();
  const int na = (nl + kMaxLattices - 1) / kMaxLattices;
  const int nb = ((int)B.size() + kMaxLattices - 1) / kMaxLattices +
                 ((int)B2.size() + kMaxLattices - 1) / kMaxLattices + (int)own.size();
  return [=](const Cx<float>* x, Cx<float>* y, int dagger, double* norm2) mutable {
    const int* act = h0->op_active;
    auto set_b = [&](LineArgs<float>& b, const JointPart& q) {
      const Cx<float>* xu = x + q.off;
      const Cx<float>* xl = xu + 6 * q.h->g.tp;
      b.src_lo = dagger ? xu : xl;
      b.active = act ? act + q.r0 : nullptr;
    };
    auto set_c = [&](LineArgs<float>& c, const JointPart& q) {
      c.xpost = x + q.off;
      c.swap_out = dagger;
      c.out = y + q.off;
      c.norm2 = norm2 ? norm2 + q.r0 : nullptr;
      c.active = act ? act + q.r0 : nullptr;
    };
    for (int j = 0; j < nl; ++j) {
      const JointPart& q = parts[j];
      const Cx<float>* xu = x + q.off;
      const Cx<float>* xl = xu + 6 * q.h->g.tp;
      A[j].src_up = dagger ? xl : xu;
      A[j].src_lo = dagger ? xu : xl;
      A[j].active = act ? act + q.r0 : nullptr;
    }
    for (size_t i = 0; i < B.size(); ++i) {
      set_b(B[i], parts[joined[i]]);
      set_c(C[i], parts[joined[i]]);
    }
    for (size_t i = 0; i < B2.size(); ++i) {
      set_b(B2[i], parts[joined2[i]]);
      set_c(C2[i], parts[joined2[i]]);
    }
    for (auto& o : own) {
      set_b(o.second.b, parts[o.first]);
      set_c(o.second.c, parts[o.first]);
    }
    cudaStream_t s = h0->stream;
    auto launch_own = [&](const Own& o, const LineArgs<float>& a, int kind) {
      if (o.t.variant == 3)
        launch_hop_pipe(a, kind, o.t.gsrc, o.t.ns, o.units, o.nunits, o.err, s);
      else
        launch_line<float>(a, kind, true, s);
    };
    { Prof P(h0, "schur_a_tdag_f32", na); launch_line_multi<float>(A, LK_SCHUR_A, s); }
    {
      Prof P(h0, "schur_b_hop_tsolve_f32", nb);
      launch_line_wide_multi<float>(B, LK_SCHUR_B, s);
      launch_line_multi<float>(B2, LK_SCHUR_B, s);
      for (const auto& o : own) launch_own(o.second, o.second.b, LK_SCHUR_B);
    }
    if (norm2) WF_CUDA(cudaMemsetAsync(norm2, 0, nr * sizeof(double), s));
    {
      Prof P(h0, "schur_c_hop_tinv_axpy_f32", nb);
      launch_line_wide_multi<float>(C, LK_SCHUR_C, s);
      launch_line_multi<float>(C2, LK_SCHUR_C, s);
      for (const auto& o : own) launch_own(o.second, o.second.c, LK_SCHUR_C);
    }
  };
}

// Temporal + 3-D Schur solve in FP32 by defect correction, for one lattice or jointly for several
// (wf_solve_many). Each pass solves M delta = r with the method's steps in FP32 -- S_L, CGNR on
// M-hat without reliable updates, S_R -- to a reduction rho of its Schur residual (no further
// than what tol needs), adds delta to the FP64 solution psi and recomputes the true residual
// r = eta - M psi in FP64, the residual the solve reports; it stops when ||r|| / ||eta|| <= tol for
// every source. The only FP64 operator apply of a pass is that true residual. h16 (WF_FP16MIX,
// one lattice): the pass's CGNR keeps its vectors in FP16 with FP32 recomputations of the
// residual (cgnr_h16 without its FP64 updates). With several
// lattices the CGNR runs over the concatenation of their odd fields (joint_schur_op) on hs[0]'s
// stream, the other steps per lattice on each handle's stream (distinct streams), so that they
// overlap; every source keeps its own CG scalars and stopping test. Environment WF_DC_RHO sets rho
// (default 1e-5).
void solve_temporal_schur_dc(int nl, wf_handle* const* hs, const std::vector<const Cx<double>*>& eta_lex,
                             const std::vector<Cx<double>*>& x_lex, const int* nrhs, double tol, bool x0,
                             std::vector<std::vector<int>>& iters, std::vector<std::vector<double>>& rel,
                             std::vector<int>& status, bool h16) {
  wf_handle* h0 = hs[0];
  cudaStream_t s = h0->stream;
  std::vector<JointPart> parts(nl);
  size_t ntot = 0, nmax = 0;
  int nr = 0;
  for (int j = 0; j < nl; ++j) {
    parts[j] = {hs[j], nrhs[j], hs[j]->half_int(), ntot, nr};
    ntot += parts[j].n * nrhs[j];
    nmax = std::max(nmax, parts[j].n);
    nr += nrhs[j];
  }
  const bool joint = nl > 1;
  if (joint && h16) throw Error(WF_EINVAL, "FP16 storage: one lattice per solve");
  const JointSync sync(parts.size());
  double rho = 1e-5;
  if (const char* e = std::getenv("WF_DC_RHO")) {
    const double v = std::atof(e);
    if (v > 0.0 && v < 1.0) rho = v;
  }
  // the solver's vectors (FP64 right-hand side and solution of the Schur system), the operator's
  // scratch fields and the first element of every source (several lattices)
  Cx<double>* b = h0->buf<Cx<double>>("sv_b_o", ntot);
  Cx<double>* y = h0->buf<Cx<double>>("sv_y_o", ntot);
  Cx<float>* ty = nullptr;
  Cx<float>* tz = nullptr;
  Cx<float>* tw = nullptr;
  size_t* offs = nullptr;
  if (joint) {
    ty = h0->buf<Cx<float>>("jv_ty_f32", ntot);
    tz = h0->buf<Cx<float>>("jv_tz_f32", ntot);
    tw = h0->buf<Cx<float>>("jv_tw_f32", ntot);
    offs = h0->buf<size_t>("jv_offs", (size_t)nr + 1);
    std::vector<size_t> o;
    for (const JointPart& q : parts)
      for (int k = 0; k < q.nrhs; ++k) o.push_back(q.off + (size_t)k * q.n);
    o.push_back(ntot);
    WF_CUDA(cudaMemcpyAsync(offs, o.data(), o.size() * sizeof(size_t), cudaMemcpyHostToDevice, s));
  }
  // o is a host temporary, and the lattices' streams write b (zeroed on s when allocated)
  WF_CUDA(cudaStreamSynchronize(s));

  struct PerLattice {
    Cx<double> *eta_e, *eta_o, *psi_e, *psi_o, *r_e, *r_o;
    Cx<float> *r32_e, *r32_o, *w32_e, *w32_o;
    double* sc;
    double* partial;
    std::vector<double> eta2;
  };
  std::vector<PerLattice> L(nl);
  // per lattice on its stream: |v_e|^2 + |v_o|^2 per source, read back after all are launched
  auto launch_norms = [&](int j, const Cx<double>* ve, const Cx<double>* vo) {
    wf_handle* h = parts[j].h;
    const int m = parts[j].nrhs;
    Prof Q(h, "norm2_f64", vo ? 4 : 2);
    launch_norm2<double>(ve, parts[j].n, m, L[j].partial, L[j].sc, h->stream);
    if (vo) launch_norm2<double>(vo, parts[j].n, m, L[j].partial, L[j].sc + m, h->stream);
  };
  auto read_norms = [&](int j, bool two) {
    const int m = parts[j].nrhs;
    const std::vector<double> v = read_scalars(parts[j].h, L[j].sc, two ? 2 * m : m);
    std::vector<double> out(m);
    for (int k = 0; k < m; ++k) out[k] = two ? v[k] + v[m + k] : v[k];
    return out;
  };
  for (int j = 0; j < nl; ++j) {
    wf_handle* h = parts[j].h;
    cudaStream_t sj = h->stream;
    const size_t nt = parts[j].n * parts[j].nrhs;
    PerLattice& P = L[j];
    P.eta_e = h->buf<Cx<double>>("sv_eta_e", nt);
    P.eta_o = h->buf<Cx<double>>("sv_eta_o", nt);
    P.psi_e = h->buf<Cx<double>>("sv_psi_e", nt);
    P.psi_o = h->buf<Cx<double>>("sv_psi_o", nt);
    P.r_e = h->buf<Cx<double>>("sv_r_e", nt);
    P.r_o = h->buf<Cx<double>>("sv_r_o", nt);
    P.r32_e = h->buf<Cx<float>>("dc_r_e", nt);
    P.r32_o = h->buf<Cx<float>>("dc_r_o", nt);
    P.w32_e = h->buf<Cx<float>>("dc_w_e", nt);
    P.w32_o = h->buf<Cx<float>>("dc_w_o", nt);
    P.sc = h->buf<double>("sv_scalars", 4 * (size_t)parts[j].nrhs);
    P.partial = h->buf<double>("cg_partial", 1024 * (size_t)parts[j].nrhs);
    { Prof Q(h, "import_spinor_f64"); launch_import_spinor<double>(h->g, eta_lex[j], P.eta_e, P.eta_o, parts[j].nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), sj); }
    launch_norms(j, P.eta_e, P.eta_o);
  }
  for (int j = 0; j < nl; ++j) L[j].eta2 = read_norms(j, true);
  for (int j = 0; j < nl; ++j) {
    wf_handle* h = parts[j].h;
    cudaStream_t sj = h->stream;
    const size_t nt = parts[j].n * parts[j].nrhs;
    PerLattice& P = L[j];
    if (x0) {
      { Prof Q(h, "import_spinor_f64"); launch_import_spinor<double>(h->g, x_lex[j], P.psi_e, P.psi_o, parts[j].nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), sj); }
      m_apply<double>(h, P.psi_e, P.psi_o, P.r_e, P.r_o, P.eta_e, P.eta_o, -1.0, parts[j].nrhs);
    } else {
      WF_CUDA(cudaMemsetAsync(P.psi_e, 0, nt * sizeof(Cx<double>), sj));
      WF_CUDA(cudaMemsetAsync(P.psi_o, 0, nt * sizeof(Cx<double>), sj));
      WF_CUDA(cudaMemcpyAsync(P.r_e, P.eta_e, nt * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, sj));
      WF_CUDA(cudaMemcpyAsync(P.r_o, P.eta_o, nt * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, sj));
    }
    launch_norms(j, P.r_e, P.r_o);
  }
  bool all_ok = true;
  for (int j = 0; j < nl; ++j) {
    const std::vector<double> r2 = read_norms(j, true);
    iters[j].assign(parts[j].nrhs, 0);
    rel[j].resize(parts[j].nrhs);
    status[j] = WF_OK;
    for (int k = 0; k < parts[j].nrhs; ++k) {
      rel[j][k] = std::sqrt(r2[k] / (L[j].eta2[k] > 0 ? L[j].eta2[k] : 1.0));
      all_ok = all_ok && rel[j][k] <= tol;
    }
  }
  const OpFn<float> A = joint ? joint_schur_op(parts, ty, tz, tw, nr) : schur_op<float>(h0, nrhs[0]);
  const OpFn<double> A64 = [](const Cx<double>*, Cx<double>*, int, double*) {
    throw Error(WF_ECUDA, "defect correction: no FP64 operator apply inside the CG");
  };
  const int maxiter = h0->maxiter;
  std::vector<double> target(nr);
  bool capped = false;
  for (int pass = 0; pass < 8 && !all_ok && !capped; ++pass) {
    // S_L in FP32 on r: w_e = C_R^e C_L^e r_e ; w_o = C_L^o [r_o + gamma_f^-1 D_s^oe w_e] -> b (FP64)
    for (int j = 0; j < nl; ++j) {
      wf_handle* h = parts[j].h;
      cudaStream_t sj = h->stream;
      const int m = parts[j].nrhs;
      const size_t nt = parts[j].n * m;
      PerLattice& P = L[j];
      Cx<double>* b_o = b + parts[j].off;
      { Prof Q(h, "d2f", 2); launch_d2f(P.r_e, P.r32_e, nt, sj); launch_d2f(P.r_o, P.r32_o, nt, sj); }
      line_load<float>(h, 0, P.r32_e, P.w32_e, OP_FWD, OP_BWD, m, "prep_tsolve");
      {
        LineArgs<float> a = line_args<float>(h, 1, m);
        a.src_up = P.w32_e;
        a.src_lo = P.w32_e + 6 * h->g.tp;
        a.xpre = P.r32_o;
        a.apre = (float)(1.0 / h->g.gamma_f);
        a.opu = OP_COPY;
        a.opl = OP_BWD;
        a.src = SRC_HOP;
        a.out = P.w32_o;
        Prof Q(h, "prep_hop_f32");
        launch_line<float>(a, LK_GENERIC, h->axial, sj);
      }
      WF_CUDA(cudaMemsetAsync(b_o, 0, nt * sizeof(Cx<double>), sj));
      { Prof Q(h, "add_f_to_d"); launch_add_f_to_d(b_o, P.w32_o, nt, sj); }
      launch_norms(j, b_o, nullptr);
    }
    // CGNR to rho ||b|| per source, no further than half of what tol needs (sources already at
    // tol start converged)
    for (int j = 0; j < nl; ++j) {
      const std::vector<double> b2 = read_norms(j, false);
      const double mu1 = parts[j].h->g.mu + 1.0;
      for (int k = 0; k < parts[j].nrhs; ++k) {
        const double bn = std::sqrt(b2[k]);
        target[parts[j].r0 + k] = rel[j][k] <= tol ? 2.0 * bn + 1.0
                                                   : std::max(rho * bn, 0.5 * tol * std::sqrt(L[j].eta2[k]) / mu1);
      }
    }
    sync.fan_in(parts);
    // the iteration limit holds for the passes together
    int used = 0;
    for (int j = 0; j < nl; ++j)
      for (int k = 0; k < parts[j].nrhs; ++k) used = std::max(used, iters[j][k]);
    const int left = std::max(1, maxiter - used);
    const std::vector<int> it =
        h16 ? cgnr_h16(h0, nr, nmax, b, y, target, left, false, false)
            : cgnr<float>(h0, A, A64, b, y, nr, nmax, target, left, false, joint ? ntot : 0, offs, false);
    sync.fan_out(parts);
    // S_R in FP32: d_o = C_R^o y_o ; d_e = C_R^e C_L^e [r_e + gamma_f^-1 D_s^eo d_o] ; psi += d ;
    // r = eta - M psi in FP64
    for (int j = 0; j < nl; ++j) {
      wf_handle* h = parts[j].h;
      cudaStream_t sj = h->stream;
      const int m = parts[j].nrhs;
      const size_t nt = parts[j].n * m;
      PerLattice& P = L[j];
      { Prof Q(h, "d2f"); launch_d2f(y + parts[j].off, P.w32_e, nt, sj); }  // y_o in FP32 (w_e is free)
      line_load<float>(h, 1, P.w32_e, P.w32_o, OP_FWD, OP_COPY, m, "recon_tsolve");
      {
        LineArgs<float> a = line_args<float>(h, 0, m);
        a.src_up = P.w32_o;
        a.src_lo = P.w32_o + 6 * h->g.tp;
        a.xpre = P.r32_e;
        a.apre = (float)(1.0 / h->g.gamma_f);
        a.opu = OP_FWD;
        a.opl = OP_BWD;
        a.src = SRC_HOP;
        a.out = P.w32_e;
        Prof Q(h, "recon_hop_f32");
        launch_line<float>(a, LK_GENERIC, h->axial, sj);
      }
      { Prof Q(h, "add_f_to_d", 2); launch_add_f_to_d(P.psi_e, P.w32_e, nt, sj); launch_add_f_to_d(P.psi_o, P.w32_o, nt, sj); }
      m_apply<double>(h, P.psi_e, P.psi_o, P.r_e, P.r_o, P.eta_e, P.eta_o, -1.0, m);
      launch_norms(j, P.r_e, P.r_o);
    }
    all_ok = true;
    for (int j = 0; j < nl; ++j) {
      const std::vector<double> r2 = read_norms(j, true);
      for (int k = 0; k < parts[j].nrhs; ++k) {
        rel[j][k] = std::sqrt(r2[k] / (L[j].eta2[k] > 0 ? L[j].eta2[k] : 1.0));
        iters[j][k] += it[parts[j].r0 + k];
        all_ok = all_ok && rel[j][k] <= tol;
        capped = capped || iters[j][k] >= maxiter;
      }
    }
  }
  for (int j = 0; j < nl; ++j) {
    wf_handle* h = parts[j].h;
    for (int k = 0; k < parts[j].nrhs; ++k)
      if (rel[j][k] > tol) status[j] = WF_ENOCONV;  // within eight passes or the iteration limit
    Prof Q(h, "export_spinor_f64");
    launch_export_spinor<double>(h->g, L[j].psi_e, L[j].psi_o, x_lex[j], parts[j].nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), h->stream);
  }
}

// Whether wf_solve_many solves its lattices jointly: on request (environment WF_JOINT=1), for FP32
// iterations of the temporal + Schur method in the axial frame, on lattices the one-thread-per-site
// kernels serve, on one device, with one iteration limit and no clover term. Measured on GB300
// (the xi sweep's three lattices; eight small lattices) the per-lattice solves on concurrent
// streams finish 10-25 % sooner: each lattice's FP64 true residuals (bound by the FP64 pipe) then
// overlap other lattices' FP32 iterations (bound by memory), while the joint passes keep every
// lattice in the same phase.
bool joint_eligible(int n, wf_handle* const* hs, int method, int precision) {
  if (n < 2 || method != WF_TEMPORAL_SCHUR || precision != WF_FP32 || !use_defect_correction()) return false;
  const char* e = std::getenv("WF_JOINT");
  if (!e || e[0] != '1') return false;
  if (const char* e = std::getenv("WF_TMA"))
    if (e[0] == '1') return false;
  for (int i = 0; i < n; ++i) {
    const wf_handle* h = hs[i];
    if (!h->gauge || h->clover || !h->axial || !wide_supported(h->g) || h->use_tma == 1) return false;
    if (h->device != hs[0]->device || h->maxiter != hs[0]->maxiter) return false;
  }
  return true;
}

// the joint solve holds every lattice's sources in one set of CG scalars
bool joint_fits(int n, const int* nrhs) {
  long long nr = 0;
  for (int i = 0; i < n; ++i) nr += nrhs[i] > 0 ? nrhs[i] : 0;
  return nr <= WF_MAX_SOLVE_RHS;
}

// wf_solve_many's joint path: argument checks and host staging per handle as in wf_solve; every
// handle works on a stream of its own (a temporary one for a handle on the default stream or on
// another handle's stream), restored after the call
void solve_many_joint(int n, wf_handle* const* hs, const double* const* rhs, double* const* x, const int* nrhs,
                      double tol, int flags, int* const* iters_out, double* const* resid_out, std::vector<int>& st) {
  std::vector<cudaStream_t> old(n), own(n, nullptr);
  for (int i = 0; i < n; ++i) old[i] = hs[i]->stream;
  int prev = 0;
  cudaGetDevice(&prev);
  auto restore = [&]() {
    for (int i = 0; i < n; ++i) {
      if (own[i]) {
        cudaStreamSynchronize(own[i]);
        cudaStreamDestroy(own[i]);
      }
      hs[i]->stream = old[i];
    }
    cudaSetDevice(prev);
  };
  try {
    for (int i = 0; i < n; ++i) hs[i]->err.clear();
    WF_CUDA(cudaSetDevice(hs[0]->device));
    if (!(tol > 0)) throw Error(WF_EINVAL, "tol must be > 0");
    for (int i = 0; i < n; ++i)
      if (nrhs[i] < 1) throw Error(WF_EINVAL, "nrhs must be >= 1");
    // work the caller queued on the handles' streams comes first
    for (int i = 0; i < n; ++i) WF_CUDA(cudaStreamSynchronize(old[i]));
    for (int i = 0; i < n; ++i) {
      bool shared = old[i] == nullptr;
      for (int j = 0; j < i && !shared; ++j) shared = old[j] == old[i];
      if (shared) {
        WF_CUDA(cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking));
        hs[i]->stream = own[i];
      }
    }
    const bool x0 = (flags & WF_X0) != 0;
    std::vector<const Cx<double>*> din(n);
    std::vector<Cx<double>*> dx(n);
    std::vector<char> staged(n);
    std::vector<size_t> le(n);
    for (int i = 0; i < n; ++i) {
      le[i] = hs[i]->lex_elems() * nrhs[i];
      din[i] = dev_in(hs[i], rhs[i], le[i], "stage_in");
      bool sg = false;
      dx[i] = dev_out(hs[i], x[i], le[i], "stage_out", sg);
      staged[i] = sg;
      if (x0 && sg)
        WF_CUDA(cudaMemcpyAsync(dx[i], x[i], le[i] * sizeof(Cx<double>), cudaMemcpyHostToDevice, hs[i]->stream));
    }
    std::vector<std::vector<int>> it(n);
    std::vector<std::vector<double>> res(n);
    solve_temporal_schur_dc(n, hs, din, dx, nrhs, tol, x0, it, res, st);
    for (int i = 0; i < n; ++i) {
      finish_out(hs[i], x[i], dx[i], le[i], staged[i]);
      for (int k = 0; k < nrhs[i]; ++k) {
        if (iters_out && iters_out[i]) iters_out[i][k] = it[i][k];
        if (resid_out && resid_out[i]) resid_out[i][k] = res[i][k];
      }
      if (st[i] == WF_ENOCONV) hs[i]->err = "solver did not reach tol";
    }
  } catch (const Error& e) {
    for (int i = 0; i < n; ++i) st[i] = fail(hs[i], e.code, e.what());
  } catch (const std::bad_alloc&) {
    for (int i = 0; i < n; ++i) st[i] = fail(hs[i], WF_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    for (int i = 0; i < n; ++i) st[i] = fail(hs[i], WF_ECUDA, e.what());
  }
  restore();
}

// ----------------------------------------------------------------------------
// Comparators: 4-D even-odd Schur, unpreconditioned M, temporal-only M~ = C_L M C_R
// ----------------------------------------------------------------------------
template <typename R>
EoArgs<R> eo_args(wf_handle* h, int par, int nrhs) {
  Gauge<R> G = gauge_of<R>(h);
  EoArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.g = h->g;
  a.par = par;
  a.nrhs = nrhs;
  for (int p = 0; p < 2; ++p) {
    a.ut[p] = G.ut[p];
    a.pl[p] = G.pl[p];
    a.us[p] = G.us[p];
  }
  a.inv_gf = (R)(1.0 / h->g.gamma_f);
  a.bc = (R)h->g.bc;
  a.a = R(1);
  a.df = (sizeof(R) == 8 && h->df_ops) ? 1 : 0;
  return a;
}

size_t eo_elems(const wf_handle* h) { return (size_t)h->g.L * h->g.L * h->g.L * NSPIN_C * (h->g.T / 2); }

template <typename R>
const Cx<R>* clover_eo(wf_handle* h, int p, bool inverse);
template <>
const Cx<double>* clover_eo<double>(wf_handle* h, int p, bool inverse) {
  return (inverse ? h->clinv64[p] : h->clmu64[p]).as<Cx<double>>();
}
template <>
const Cx<float>* clover_eo<float>(wf_handle* h, int p, bool inverse) {
  return (inverse ? h->clinv32[p] : h->clmu32[p]).as<Cx<float>>();
}

// out = acc + alpha (mu + A)^pp in, or with (mu + A)^-1 (inverse), on 4-D even-odd fields
template <typename R>
void clover_eo_on(wf_handle* h, int p, bool inverse, const Cx<R>* in, Cx<R>* out, const Cx<R>* acc, double alpha,
                  int nrhs) {
  Prof P(h, pname<R>(inverse ? "clover_inv_eo" : "clover_mu_eo"));
  launch_clover_apply_eo<R>(h->g, clover_eo<R>(h, p, inverse), in, out, acc, alpha, nrhs, h->stream);
}

// M-hat_4 = mu - mu^-1 D_w^oe D_w^eo on odd 4-D fields (dagger: S M-hat_4 S), two dslash kernels;
// with a clover term (mu + A)^oo - D_w^oe (mu + A)^-1_ee D_w^eo (mu + A commutes with gamma_5, so
// the adjoint exchanges spin halves only around the dslash terms)
template <typename R>
void eo4d_apply(wf_handle* h, const Cx<R>* x, Cx<R>* out, int dagger, int nrhs, Cx<R>* he, double* norm2) {
  const double mu = h->g.mu;
  if (h->clover) {
    const size_t nt = eo_elems(h) * nrhs;
    Cx<R>* he2 = h->buf<Cx<R>>(pname<R>("op_he2"), nt);
    Cx<R>* tx = h->buf<Cx<R>>(pname<R>("op_tx"), nt);
    {
      EoArgs<R> a = eo_args<R>(h, 0, nrhs);
      a.in = x;
      a.swap_in = dagger;
      a.out = he;
      Prof P(h, pname<R>("eo4d_dslash_eo"));
      launch_dslash4<R>(a, h->axial, h->stream);
    }
    clover_eo_on<R>(h, 0, true, he, he2, nullptr, 1.0, nrhs);
    clover_eo_on<R>(h, 1, false, x, tx, nullptr, 1.0, nrhs);
    EoArgs<R> a = eo_args<R>(h, 1, nrhs);
    a.in = he2;
    a.a = R(-1);
    a.x1 = tx;
    a.b1 = R(1);
    a.swap_out = dagger;
    a.stream_out = 1;
    a.out = out;
    a.norm2 = norm2;
    if (norm2) WF_CUDA(cudaMemsetAsync(norm2, 0, nrhs * sizeof(double), h->stream));
    Prof P(h, pname<R>("eo4d_dslash_oe_axpy"));
    launch_dslash4<R>(a, h->axial, h->stream);
    return;
  }
  {
    EoArgs<R> a = eo_args<R>(h, 0, nrhs);
    a.in = x;
    a.swap_in = dagger;
    a.out = he;
    Prof P(h, pname<R>("eo4d_dslash_eo"));
    launch_dslash4<R>(a, h->axial, h->stream);
  }
  {
    EoArgs<R> a = eo_args<R>(h, 1, nrhs);
    a.in = he;
    a.a = (R)(-1.0 / mu);
    a.x1 = x;
    a.b1 = (R)mu;
    a.swap_out = dagger;
    a.stream_out = 1;  // the operator's result is next read by the solver's vector update
    a.out = out;
    a.norm2 = norm2;
    if (norm2) WF_CUDA(cudaMemsetAsync(norm2, 0, nrhs * sizeof(double), h->stream));
    Prof P(h, pname<R>("eo4d_dslash_oe_axpy"));
    launch_dslash4<R>(a, h->axial, h->stream);
  }
}

template <typename R>
OpFn<R> eo4d_op(wf_handle* h, int nrhs) {
  Cx<R>* he = h->buf<Cx<R>>(pname<R>("op_he"), eo_elems(h) * nrhs);
  return [=](const Cx<R>* x, Cx<R>* y, int dagger, double* norm2) { eo4d_apply<R>(h, x, y, dagger, nrhs, he, norm2); };
}

std::vector<double> eo_norms(wf_handle* h, const Cx<double>* a, const Cx<double>* b, size_t n, int nrhs) {
  double* sc = h->buf<double>("sv_scalars", 4 * (size_t)nrhs);
  double* partial = h->buf<double>("cg_partial", 1024 * (size_t)nrhs);
  {
    Prof P(h, "norm2_f64", 4);
    launch_norm2<double>(a, n, nrhs, partial, sc, h->stream);
    launch_norm2<double>(b, n, nrhs, partial, sc + nrhs, h->stream);
  }
  std::vector<double> v = read_scalars(h, sc, 2 * nrhs), out(nrhs);
  for (int k = 0; k < nrhs; ++k) out[k] = v[k] + v[nrhs + k];
  return out;
}

// Standard 4-D even-odd solve (§II.B, 4D-Schur): b_o = eta_o + mu^-1 D_w^oe eta_e, CGNR on
// M-hat_4, psi_e = mu^-1 (eta_e + D_w^eo psi_o); true residual with M = mu - D_w.
int solve_eo4d(wf_handle* h, const Cx<double>* eta_lex, Cx<double>* x_lex, int nrhs, double tol, int precision,
               bool x0, int* iters_out, double* resid_out) {
  if (h->g.T % 2) throw Error(WF_EINVAL, "the 4-D even-odd method needs an even T");
  const size_t n = eo_elems(h), nt = n * nrhs;
  cudaStream_t s = h->stream;
  DfScope dfs(h, precision == WF_FP32);
  const double mu = h->g.mu;
  Cx<double>* eta_e = h->buf<Cx<double>>("eo_eta_e", nt);
  Cx<double>* eta_o = h->buf<Cx<double>>("eo_eta_o", nt);
  Cx<double>* b_o = h->buf<Cx<double>>("eo_b_o", nt);
  Cx<double>* psi_e = h->buf<Cx<double>>("eo_psi_e", nt);
  Cx<double>* psi_o = h->buf<Cx<double>>("eo_psi_o", nt);
  Cx<double>* r_e = h->buf<Cx<double>>("eo_r_e", nt);
  Cx<double>* r_o = h->buf<Cx<double>>("eo_r_o", nt);
  {
    Prof P(h, "import_eo_f64");
    launch_import_eo<double>(h->g, eta_lex, eta_e, eta_o, nrhs, frame_rot(h, 0), frame_rot(h, 1), -1, s);
  }
  const bool cl = h->clover;  // clover: (mu + A)^-1_ee in place of mu^-1, (mu + A) psi in the residual
  if (cl) clover_eo_on<double>(h, 0, true, eta_e, r_e, nullptr, 1.0, nrhs);  // r_e = (mu + A)^-1 eta_e
  {
    EoArgs<double> a = eo_args<double>(h, 1, nrhs);
    a.in = cl ? r_e : eta_e;
    a.a = cl ? 1.0 : 1.0 / mu;
    a.x1 = eta_o;
    a.b1 = 1.0;
    a.out = b_o;
    Prof P(h, "eo4d_prep_f64");
    launch_dslash4<double>(a, h->axial, s);
  }
  if (x0) {
    Prof P(h, "import_eo_f64");
    launch_import_eo<double>(h->g, x_lex, r_e, psi_o, nrhs, frame_rot(h, 0), frame_rot(h, 1), -1, s);
  }
  std::vector<double> eta2 = eo_norms(h, eta_e, eta_o, n, nrhs), target(nrhs);
  for (int k = 0; k < nrhs; ++k) target[k] = tol * std::sqrt(eta2[k]);  // |eta - M psi| = |b_o - M-hat_4 psi_o|
  std::vector<int> iters(nrhs, 0);
  std::vector<double> rel(nrhs, 0.0);
  const int maxiter = h->maxiter;
  int status = WF_OK;
  bool have_x0 = x0;
  for (int pass = 0; pass < 6; ++pass) {
    std::vector<int> it = precision == WF_FP32
                              ? cgnr<float>(h, eo4d_op<float>(h, nrhs), eo4d_op<double>(h, nrhs), b_o, psi_o, nrhs, n,
                                            target, maxiter, have_x0)
                              : cgnr<double>(h, eo4d_op<double>(h, nrhs), eo4d_op<double>(h, nrhs), b_o, psi_o, nrhs,
                                             n, target, maxiter, have_x0);
    for (int k = 0; k < nrhs; ++k) iters[k] += it[k];
    have_x0 = true;
    {
      EoArgs<double> a = eo_args<double>(h, 0, nrhs);  // psi_e = mu^-1 (eta_e + D_w^eo psi_o)
      a.in = psi_o;
      a.a = cl ? 1.0 : 1.0 / mu;
      a.x1 = eta_e;
      a.b1 = cl ? 1.0 : 1.0 / mu;
      a.out = cl ? r_e : psi_e;
      Prof P(h, "eo4d_recon_f64");
      launch_dslash4<double>(a, h->axial, s);
    }
    if (cl) clover_eo_on<double>(h, 0, true, r_e, psi_e, nullptr, 1.0, nrhs);  // psi_e = (mu + A)^-1 (...)
    for (int p = 0; p < 2; ++p) {  // r = eta - mu psi + D_w psi (clover: eta - (mu + A) psi + D_w psi)
      Cx<double>* rp = p ? r_o : r_e;
      const Cx<double>* own = p ? psi_o : psi_e;
      if (cl) clover_eo_on<double>(h, p, false, own, rp, nullptr, 1.0, nrhs);  // r_p = (mu + A) psi_p
      EoArgs<double> a = eo_args<double>(h, p, nrhs);
      a.in = p ? psi_e : psi_o;
      a.a = 1.0;
      a.x1 = p ? eta_o : eta_e;
      a.b1 = 1.0;
      a.x2 = cl ? rp : own;
      a.b2 = cl ? -1.0 : -mu;
      a.out = rp;
      a.df = 0;  // the true residual in FP64 arithmetic
      Prof P(h, "eo4d_residual_f64");
      launch_dslash4<double>(a, h->axial, s);
    }
    std::vector<double> r2 = eo_norms(h, r_e, r_o, n, nrhs);
    bool ok = true;
    for (int k = 0; k < nrhs; ++k) {
      rel[k] = std::sqrt(r2[k] / (eta2[k] > 0 ? eta2[k] : 1.0));
      if (rel[k] > tol) {
        ok = false;
        target[k] *= 0.5 * tol / rel[k];
      }
      if (iters[k] >= maxiter) status = WF_ENOCONV;
    }
    if (ok || status == WF_ENOCONV) break;
    if (pass == 5) status = WF_ENOCONV;
  }
  {
    Prof P(h, "export_eo_f64");
    launch_export_eo<double>(h->g, psi_e, psi_o, x_lex, nrhs, frame_rot(h, 0), frame_rot(h, 1), -1, s);
  }
  for (int k = 0; k < nrhs; ++k) {
    if (iters_out) iters_out[k] = iters[k];
    if (resid_out) resid_out[k] = rel[k];
  }
  return status;
}

// Full-lattice operators (one right-hand side; a vector is [even half][odd half] of the line
// layout): M (unpreconditioned) and M~ = C_L M C_R (temporal only, §II.A). Daggers use
// gamma_5-hermiticity, M^dag = S M S and M~^dag = S M~ S with S the spin-half exchange.
template <typename R>
OpFn<R> full_op(wf_handle* h, bool temporal) {
  const size_t hn = h->half_int();
  Cx<R>* t1 = h->buf<Cx<R>>(pname<R>("op_t1"), 2 * hn);
  Cx<R>* t2 = h->buf<Cx<R>>(pname<R>("op_t2"), 2 * hn);
  double* partial = h->buf<double>("op_partial", 1024);
  return [=](const Cx<R>* x, Cx<R>* y, int dagger, double* norm2) {
    const int tp = h->g.tp;
    auto mrun = [&](const Cx<R>* in, Cx<R>* out, int swap) {
      Gauge<R> G = gauge_of<R>(h);
      for (int p = 0; p < 2; ++p) {
        MArgs<R> m;
        std::memset(&m, 0, sizeof(m));
        m.g = h->g;
        m.parity = p;
        m.nrhs = 1;
        m.psi_p = in + p * hn;
        m.psi_q = in + (1 - p) * hn;
        m.ut = G.ut[p];
        m.pl = G.pl[p];
        m.us_out = G.us[p];
        m.us_nbr = G.us[1 - p];
        m.swap = swap;
        m.out = out + p * hn;
        m.mu = (R)h->g.mu;
        m.inv_gf = (R)(1.0 / h->g.gamma_f);
        m.bc = (R)h->g.bc;
        Prof P(h, pname<R>("apply_M"));
        launch_apply_M<R>(m, h->axial, h->stream);
      }
    };
    if (!temporal) {
      mrun(x, y, dagger);
    } else {
      // C_R (reading the halves exchanged for the dagger), M, C_L (writing them exchanged)
      for (int p = 0; p < 2; ++p) {
        LineArgs<R> a = line_args<R>(h, p, 1);
        a.src_up = x + p * hn + (dagger ? 6 * tp : 0);
        a.src_lo = x + p * hn + (dagger ? 0 : 6 * tp);
        a.opu = OP_FWD;
        a.opl = OP_COPY;
        a.src = SRC_LOAD;
        a.out = t1 + p * hn;
        Prof P(h, pname<R>("c_right"));
        launch_line<R>(a, LK_GENERIC, h->axial, h->stream);
      }
      mrun(t1, t2, 0);
      for (int p = 0; p < 2; ++p) {
        LineArgs<R> a = line_args<R>(h, p, 1);
        a.src_up = t2 + p * hn;
        a.src_lo = t2 + p * hn + 6 * tp;
        a.opu = OP_COPY;
        a.opl = OP_BWD;
        a.src = SRC_LOAD;
        a.swap_out = dagger;
        a.out = y + p * hn;
        Prof P(h, pname<R>("c_left"));
        launch_line<R>(a, LK_GENERIC, h->axial, h->stream);
      }
    }
    if (norm2) {
      Prof P(h, pname<R>("norm2"), 2);
      launch_norm2<R>(y, 2 * hn, 1, partial, norm2, h->stream);
    }
  };
}

// Unpreconditioned (CGNR on M) or temporal-only (CGNR on C_L M C_R, source C_L eta, solution
// C_R y) solve, one right-hand side at a time.
int solve_full(wf_handle* h, const Cx<double>* eta_lex, Cx<double>* x_lex, int nrhs, double tol, int precision,
               bool x0, bool temporal, int* iters_out, double* resid_out) {
  const size_t hn = h->half_int(), le = h->lex_elems();
  cudaStream_t s = h->stream;
  DfScope dfs(h, precision == WF_FP32);
  Cx<double>* eta = h->buf<Cx<double>>("fu_eta", 2 * hn);
  Cx<double>* b = h->buf<Cx<double>>("fu_b", 2 * hn);
  Cx<double>* y = h->buf<Cx<double>>("fu_y", 2 * hn);
  Cx<double>* psi = h->buf<Cx<double>>("fu_psi", 2 * hn);
  Cx<double>* r = h->buf<Cx<double>>("fu_r", 2 * hn);
  const double cl_bound = temporal ? 1.0 + h->g.mu : 1.0;  // |C_L^-1| <= 1 + mu
  int status = WF_OK;
  for (int k = 0; k < nrhs; ++k) {
    {
      Prof P(h, "import_spinor_f64");
      launch_import_spinor<double>(h->g, eta_lex + k * le, eta, eta + hn, 1, 0, frame_rot(h, 0), frame_rot(h, 1), s);
    }
    if (temporal) {
      line_load<double>(h, 0, eta, b, OP_COPY, OP_BWD, 1, "c_left");
      line_load<double>(h, 1, eta + hn, b + hn, OP_COPY, OP_BWD, 1, "c_left");
    } else {
      WF_CUDA(cudaMemcpyAsync(b, eta, 2 * hn * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, s));
    }
    if (x0) {
      Prof P(h, "import_spinor_f64");
      launch_import_spinor<double>(h->g, x_lex + k * le, y, y + hn, 1, 0, frame_rot(h, 0), frame_rot(h, 1), s);
    }
    std::vector<double> eta2 = eo_norms(h, eta, eta + hn, hn, 1);
    std::vector<double> target{tol * std::sqrt(eta2[0]) / cl_bound};
    int its = 0;
    double rel = 0.0;
    bool have_x0 = x0;
    for (int pass = 0; pass < 6; ++pass) {
      std::vector<int> it = precision == WF_FP32
                                ? cgnr<float>(h, full_op<float>(h, temporal), full_op<double>(h, temporal), b, y, 1,
                                              2 * hn, target, h->maxiter, have_x0)
                                : cgnr<double>(h, full_op<double>(h, temporal), full_op<double>(h, temporal), b, y, 1,
                                               2 * hn, target, h->maxiter, have_x0);
      its += it[0];
      have_x0 = true;
      if (temporal) {
        line_load<double>(h, 0, y, psi, OP_FWD, OP_COPY, 1, "c_right");
        line_load<double>(h, 1, y + hn, psi + hn, OP_FWD, OP_COPY, 1, "c_right");
      } else {
        WF_CUDA(cudaMemcpyAsync(psi, y, 2 * hn * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, s));
      }
      m_apply<double>(h, psi, psi + hn, r, r + hn, eta, eta + hn, -1.0, 1);
      std::vector<double> r2 = eo_norms(h, r, r + hn, hn, 1);
      rel = std::sqrt(r2[0] / (eta2[0] > 0 ? eta2[0] : 1.0));
      if (rel <= tol) break;
      if (its >= h->maxiter || pass == 5) {
        status = WF_ENOCONV;
        break;
      }
      target[0] *= 0.5 * tol / rel;
    }
    {
      Prof P(h, "export_spinor_f64");
      launch_export_spinor<double>(h->g, psi, psi + hn, x_lex + k * le, 1, 0, frame_rot(h, 0), frame_rot(h, 1), s);
    }
    if (iters_out) iters_out[k] = its;
    if (resid_out) resid_out[k] = rel;
  }
  return status;
}

// ----------------------------------------------------------------------------
// Clover (SW) operator M_SW = M + A with partial temporal preconditioning and 3-D ILU
// (§II.B, Eq. TPrecPartial; App. B): the Wilson C_L, C_R and S_L, S_R applied to M_SW give
//   M-tilde_ILU = [[1 + Abar^ee, g Abar^ee Dbar^eo], [g Dbar^oe Abar^ee, 1 + Abar^oo - g^2 Dbar^oe (1 - Abar^ee) Dbar^eo]],
// g = 1/gamma_f, Abar = C_L A C_R, Dbar = C_L D_s C_R; M_SW psi = eta is solved as
// M-tilde_ILU y = S_L eta, psi = S_R y. Without a clover term A = 0 and M-tilde_ILU = diag(1, M-hat).
// ----------------------------------------------------------------------------

template <typename R>
const Cx<R>* clover_blocks(wf_handle* h, int p);
template <>
const Cx<double>* clover_blocks<double>(wf_handle* h, int p) {
  return h->clov64[p].as<Cx<double>>();
}
template <>
const Cx<float>* clover_blocks<float>(wf_handle* h, int p) {
  return h->clov32[p].as<Cx<float>>();
}

// out = D_s^{par_out, 1 - par_out} in
template <typename R>
void hop_to(wf_handle* h, int par_out, const Cx<R>* in, Cx<R>* out, const char* name) {
  LineArgs<R> a = line_args<R>(h, par_out, 1);
  a.src_up = in;
  a.src_lo = in + 6 * h->g.tp;
  a.opu = OP_COPY;
  a.opl = OP_COPY;
  a.src = SRC_HOP;
  a.out = out;
  Prof P(h, pname<R>(name));
  launch_line<R>(a, LK_GENERIC, h->axial, h->stream);
}

// out = acc + alpha A^pp in
template <typename R>
void clover_on(wf_handle* h, int p, const Cx<R>* in, Cx<R>* out, const Cx<R>* acc, double alpha, int nrhs) {
  Prof P(h, pname<R>("clover_apply"));
  launch_clover_apply<R>(h->g, clover_blocks<R>(h, p), in, out, acc, alpha, nrhs, h->stream);
}

// out = xpost + apost C[xpre + apre S(in)] on the lines of `parity` for one right-hand side: S the
// site's own spinor (SRC_LOAD) or D_s of the other parity (SRC_HOP), C the line operation opu /
// opl per spin half; xpre / xpost null: no pre- / post-axpy
template <typename R>
void line_step(wf_handle* h, int parity, int src, const Cx<R>* in, Cx<R>* out, int opu, int opl, const Cx<R>* xpre,
               double apre, const Cx<R>* xpost, double apost, const char* name) {
  LineArgs<R> a = line_args<R>(h, parity, 1);
  a.src = src;
  a.src_up = in;
  a.src_lo = in + 6 * h->g.tp;
  a.opu = opu;
  a.opl = opl;
  a.xpre = xpre;
  a.apre = (R)apre;
  a.xpost = xpost;
  a.apost = (R)apost;
  a.out = out;
  // a hop followed by C_L has the compiled variant of the Schur operator's K-c (in FP32 in the
  // axial frame: the one-thread-per-site kernel)
  const int kind = src == SRC_HOP && opu == OP_COPY && opl == OP_BWD ? LK_SCHUR_C : LK_GENERIC;
  Prof P(h, pname<R>(name));
  launch_line<R>(a, kind, h->axial, h->stream);
}

// chi = M-tilde_ILU psi for one right-hand side, by the sequence of App. B
//   t1 = g Dbar^eo psi_o, t2 = Abar^ee (t1 + psi_e), chi_e = psi_e + t2,
//   chi_o = psi_o + Abar^oo psi_o + g Dbar^oe (t2 - t1)
// (g = 1 / gamma_f, Dbar = C_L D_s C_R, Abar = C_L A C_R), with each line operation's axpys folded
// into its kernel: with a = C_R^o psi_o and u = C_L^e D_s^eo a (so t1 = g u),
//   t2 = C_L^e A^ee C_R^e (psi_e + g u),  chi_e = psi_e + t2,
//   chi_o = [psi_o + C_L^o A^oo a] + g C_L^o D_s^oe C_R^e (t2 - g u);
// without a clover term t2 = 0 and chi_o = psi_o - g^2 C_L^o D_s^oe C_R^e u.
template <typename R>
void ilu_apply(wf_handle* h, const Cx<R>* pe, const Cx<R>* po, Cx<R>* ce, Cx<R>* co) {
  const size_t hn = h->half_int();
  cudaStream_t s = h->stream;
  const double g = 1.0 / h->g.gamma_f;
  Cx<R>* a = h->buf<Cx<R>>(pname<R>("il_a"), hn);
  Cx<R>* u = h->buf<Cx<R>>(pname<R>("il_u"), hn);
  Cx<R>* c = h->buf<Cx<R>>(pname<R>("il_c"), hn);
  Cx<R>* d = h->buf<Cx<R>>(pname<R>("il_d"), hn);
  Cx<R>* t2 = h->buf<Cx<R>>(pname<R>("il_t2"), hn);
  Cx<R>* e = h->buf<Cx<R>>(pname<R>("il_e"), hn);
  line_step<R>(h, 1, SRC_LOAD, po, a, OP_FWD, OP_COPY, nullptr, 0.0, nullptr, 0.0, "il_c_right");  // a = C_R^o psi_o
  line_step<R>(h, 0, SRC_HOP, a, u, OP_COPY, OP_BWD, nullptr, 0.0, nullptr, 0.0, "il_hop_c_left");  // u = C_L^e D a
  if (h->clover) {
    line_step<R>(h, 0, SRC_LOAD, u, c, OP_FWD, OP_COPY, pe, g, nullptr, 0.0, "il_c_right");  // C_R^e (psi_e + g u)
    clover_on<R>(h, 0, c, d, nullptr, 1.0, 1);
    line_step<R>(h, 0, SRC_LOAD, d, t2, OP_COPY, OP_BWD, nullptr, 0.0, nullptr, 0.0, "il_c_left");  // t2
    line_step<R>(h, 0, SRC_LOAD, t2, ce, OP_COPY, OP_COPY, pe, 1.0, nullptr, 0.0, "il_axpy");  // chi_e = psi_e + t2
    line_step<R>(h, 0, SRC_LOAD, u, c, OP_FWD, OP_COPY, t2, -g, nullptr, 0.0, "il_c_right");  // C_R^e (t2 - g u)
    clover_on<R>(h, 1, a, d, nullptr, 1.0, 1);  // d = A^oo C_R^o psi_o
    line_step<R>(h, 1, SRC_LOAD, d, e, OP_COPY, OP_BWD, nullptr, 0.0, po, 1.0, "il_c_left");  // psi_o + Abar^oo psi_o
    line_step<R>(h, 1, SRC_HOP, c, co, OP_COPY, OP_BWD, nullptr, 0.0, e, g, "il_hop_c_left");
  } else {
    WF_CUDA(cudaMemcpyAsync(ce, pe, hn * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, s));
    line_step<R>(h, 0, SRC_LOAD, u, c, OP_FWD, OP_COPY, nullptr, 0.0, nullptr, 0.0, "il_c_right");  // C_R^e u
    line_step<R>(h, 1, SRC_HOP, c, co, OP_COPY, OP_BWD, nullptr, 0.0, po, -g * g, "il_hop_c_left");
  }
}

// M-tilde_ILU on [even | odd] internal vectors (one right-hand side); the adjoint is
// gamma_5 M-tilde_ILU gamma_5 (S_R^dag = gamma_5 S_L gamma_5, M_SW gamma_5-hermitian), applied
// with the spin halves exchanged on both sides
template <typename R>
OpFn<R> ilu_op(wf_handle* h) {
  return [=](const Cx<R>* x, Cx<R>* y, int dagger, double* norm2) {
    const size_t hn = h->half_int();
    cudaStream_t s = h->stream;
    if (dagger) {
      Cx<R>* xs = h->buf<Cx<R>>(pname<R>("il_xs"), 2 * hn);
      Cx<R>* ys = h->buf<Cx<R>>(pname<R>("il_ys"), 2 * hn);
      {
        Prof P(h, pname<R>("il_swap"));
        launch_swap_halves<R>(x, xs, 2 * hn, h->g.tp, s);
      }
      ilu_apply<R>(h, xs, xs + hn, ys, ys + hn);
      Prof P(h, pname<R>("il_swap"));
      launch_swap_halves<R>(ys, y, 2 * hn, h->g.tp, s);
    } else {
      ilu_apply<R>(h, x, x + hn, y, y + hn);
    }
    if (norm2) {
      double* partial = h->buf<double>("op_partial", 1024);
      Prof P(h, pname<R>("norm2"), 2);
      launch_norm2<R>(y, 2 * hn, 1, partial, norm2, s);
    }
  };
}

// M_SW psi = eta for each right-hand side: b = S_L eta, CGNR on M-tilde_ILU y = b, psi = S_R y,
// accepted on the FP64 true residual of M_SW (the inner target tightened until it is met)
int solve_temporal_ilu(wf_handle* h, const Cx<double>* eta_lex, Cx<double>* x_lex, int nrhs, double tol,
                       int precision, int* iters_out, double* resid_out) {
  const size_t hn = h->half_int(), le = h->lex_elems();
  cudaStream_t s = h->stream;
  DfScope dfs(h, precision == WF_FP32);
  const double g = 1.0 / h->g.gamma_f;
  Cx<double>* eta = h->buf<Cx<double>>("tl_eta", 2 * hn);
  Cx<double>* b = h->buf<Cx<double>>("tl_b", 2 * hn);
  Cx<double>* y = h->buf<Cx<double>>("tl_y", 2 * hn);
  Cx<double>* psi = h->buf<Cx<double>>("tl_psi", 2 * hn);
  Cx<double>* r = h->buf<Cx<double>>("tl_r", 2 * hn);
  Cx<double>* u = h->buf<Cx<double>>("tl_u", hn);
  Cx<double>* v = h->buf<Cx<double>>("tl_v", hn);
  auto axpby = [&](Cx<double>* yy, const Cx<double>* xx, double al, double be) {
    Prof P(h, "tl_axpby_f64");
    launch_axpby<double>(yy, xx, hn, al, be, s);
  };
  int status = WF_OK;
  for (int k = 0; k < nrhs; ++k) {
    {
      Prof P(h, "import_spinor_f64");
      launch_import_spinor<double>(h->g, eta_lex + k * le, eta, eta + hn, 1, 0, frame_rot(h, 0), frame_rot(h, 1), s);
    }
    // b = S_L eta: b_e = C_L^e eta_e, b_o = C_L^o (eta_o + g D_s^oe C_R^e b_e)
    line_load<double>(h, 0, eta, b, OP_COPY, OP_BWD, 1, "tl_c_left");
    line_load<double>(h, 0, b, u, OP_FWD, OP_COPY, 1, "tl_c_right");
    hop_to<double>(h, 1, u, v, "tl_hop");
    axpby(v, eta + hn, 1.0, g);
    line_load<double>(h, 1, v, b + hn, OP_COPY, OP_BWD, 1, "tl_c_left");
    std::vector<double> eta2 = eo_norms(h, eta, eta + hn, hn, 1);
    std::vector<double> target{tol * std::sqrt(eta2[0]) / (1.0 + h->g.mu)};
    int its = 0;
    double rel = 0.0;
    bool have_x0 = false;
    for (int pass = 0; pass < 6; ++pass) {
      std::vector<int> it = precision == WF_FP32
                                ? cgnr<float>(h, ilu_op<float>(h), ilu_op<double>(h), b, y, 1, 2 * hn, target, h->maxiter,
                                              have_x0)
                                : cgnr<double>(h, ilu_op<double>(h), ilu_op<double>(h), b, y, 1, 2 * hn, target,
                                               h->maxiter, have_x0);
      its += it[0];
      have_x0 = true;
      // psi = S_R y: psi_o = C_R^o y_o, psi_e = C_R^e (y_e + g C_L^e D_s^eo C_R^o y_o)
      line_load<double>(h, 1, y + hn, psi + hn, OP_FWD, OP_COPY, 1, "tl_c_right");
      hop_to<double>(h, 0, psi + hn, u, "tl_hop");
      line_load<double>(h, 0, u, v, OP_COPY, OP_BWD, 1, "tl_c_left");
      axpby(v, y, 1.0, g);
      line_load<double>(h, 0, v, psi, OP_FWD, OP_COPY, 1, "tl_c_right");
      // r = eta - M_SW psi
      m_apply<double>(h, psi, psi + hn, r, r + hn, eta, eta + hn, -1.0, 1);
      if (h->clover) {
        clover_on<double>(h, 0, psi, r, r, -1.0, 1);
        clover_on<double>(h, 1, psi + hn, r + hn, r + hn, -1.0, 1);
      }
      std::vector<double> r2 = eo_norms(h, r, r + hn, hn, 1);
      rel = std::sqrt(r2[0] / (eta2[0] > 0 ? eta2[0] : 1.0));
      if (rel <= tol) break;
      if (its >= h->maxiter || pass == 5) {
        status = WF_ENOCONV;
        break;
      }
      target[0] *= 0.5 * tol / rel;
    }
    {
      Prof P(h, "export_spinor_f64");
      launch_export_spinor<double>(h->g, psi, psi + hn, x_lex + k * le, 1, 0, frame_rot(h, 0), frame_rot(h, 1), s);
    }
    if (iters_out) iters_out[k] = its;
    if (resid_out) resid_out[k] = rel;
  }
  return status;
}

// ----------------------------------------------------------------------------
// Pseudofermion force (HMC use of the preconditioner, proposed in §IV)
// ----------------------------------------------------------------------------

// CG on the normal operator A^dag A x = b in precision R (FP64 reliable updates for R = float);
// stops when |b - A^dag A x| <= tol |b|. One right-hand side. Returns the iterations.
template <typename R>
int cg_normal(wf_handle* h, const OpFn<R>& A, const OpFn<double>& A64, const Cx<double>* b, Cx<double>* x, size_t n,
              double tol, int maxiter) {
  cudaStream_t s = h->stream;
  double* sc = h->buf<double>("cn_scalars", 8);
  double *rr = sc, *rrn = sc + 1, *tt = sc + 2, *b2 = sc + 3;
  int* active = h->buf<int>("cg_active", 1);
  double* partial = h->buf<double>("cg_partial", 1024);
  const int one = 1;
  WF_CUDA(cudaMemcpyAsync(active, &one, sizeof(int), cudaMemcpyHostToDevice, s));
  Cx<R>* r = h->buf<Cx<R>>(pname<R>("cn_r"), n);
  Cx<R>* p = h->buf<Cx<R>>(pname<R>("cn_p"), n);
  Cx<R>* t = h->buf<Cx<R>>(pname<R>("cn_t"), n);
  Cx<R>* q = h->buf<Cx<R>>(pname<R>("cn_q"), n);
  Cx<R>* xi = h->buf<Cx<R>>(pname<R>("cn_x"), n);
  Cx<double>* r64 = h->buf<Cx<double>>("cn_r64", n);
  Cx<double>* t64 = h->buf<Cx<double>>("cn_t64", n);
  const bool mixed = sizeof(R) == 4;
  WF_CUDA(cudaMemsetAsync(x, 0, n * sizeof(Cx<double>), s));
  WF_CUDA(cudaMemsetAsync(xi, 0, n * sizeof(Cx<R>), s));
  Cx<R>* xacc = mixed ? xi : reinterpret_cast<Cx<R>*>(x);
  if (mixed) {
    Prof P(h, "d2f");
    launch_d2f(b, reinterpret_cast<Cx<float>*>(r), n, s);
  } else {
    WF_CUDA(cudaMemcpyAsync(r, b, n * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, s));
  }
  WF_CUDA(cudaMemcpyAsync(p, r, n * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, s));
  {
    Prof P(h, "norm2_f64", 2);
    launch_norm2<double>(b, n, 1, partial, b2, s);
  }
  WF_CUDA(cudaMemcpyAsync(rr, b2, sizeof(double), cudaMemcpyDeviceToDevice, s));
  const double bn2 = read_scalars(h, b2, 1)[0];
  const double target2 = tol * tol * bn2;
  double rmax = std::sqrt(bn2);
  double delta = 1e-4;
  if (const char* e = std::getenv("WF_RELIABLE_DELTA")) {
    const double v = std::atof(e);
    if (v > 0.0 && v < 1.0) delta = v;
  }
  int it = 0;
  if (bn2 == 0.0) return 0;
  for (; it < maxiter; ++it) {
    A(p, t, 0, tt);       // t = A p, |t|^2 = <p, A^dag A p>
    A(t, q, 1, nullptr);  // q = A^dag A p
    {
      Prof P(h, pname<R>("cg_xr"), 2);
      launch_cg_xr<R>(xacc, r, p, q, n, 1, rr, tt, active, partial, rrn, s);
    }
    const double rn2 = read_scalars(h, rrn, 1)[0];
    bool done = false;
    if (mixed && (std::sqrt(rn2) < delta * rmax || rn2 <= target2)) {
      {
        Prof P(h, "add_f_to_d");
        launch_add_f_to_d(x, reinterpret_cast<const Cx<float>*>(xi), n, s);
      }
      WF_CUDA(cudaMemsetAsync(xi, 0, n * sizeof(Cx<R>), s));
      A64(x, t64, 0, nullptr);
      A64(t64, r64, 1, nullptr);
      {
        Prof P(h, "axpby_f64");
        launch_axpby<double>(r64, b, n, 1.0, -1.0, s);
      }
      {
        Prof P(h, "norm2_f64", 2);
        launch_norm2<double>(r64, n, 1, partial, rrn, s);
      }
      {
        Prof P(h, "d2f");
        launch_d2f(r64, reinterpret_cast<Cx<float>*>(r), n, s);
      }
      const double t2 = read_scalars(h, rrn, 1)[0];
      rmax = std::sqrt(t2);
      done = t2 <= target2;
    } else if (!mixed) {
      done = rn2 <= target2;
    }
    if (done) {
      ++it;
      break;
    }
    {
      Prof P(h, pname<R>("cg_p"));
      launch_cg_p<R>(p, r, n, 1, rrn, rr, active, s);
    }
    {
      Prof P(h, "copy_scalar");
      launch_copy_scalar(rr, rrn, 1, s);
    }
  }
  if (mixed) {
    Prof P(h, "add_f_to_d");
    launch_add_f_to_d(x, reinterpret_cast<const Cx<float>*>(xi), n, s);
  }
  return it;
}

int force_abi(wf_handle* h, const double* phi_odd, double* F, int precision, double tol, double* action,
              int* iters_out) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (h->clover) throw Error(WF_EINVAL, "the force is that of the Wilson operator: load the gauge field without a clover term");
  if (!(tol > 0)) throw Error(WF_EINVAL, "tol must be > 0");
  const Geom& g = h->g;
  const size_t n = h->half_int();
  const size_t V = (size_t)g.L * g.L * g.L * g.T;
  const size_t ce = V / 2 * NSPIN_C;
  cudaStream_t s = h->stream;
  const Cx<double>* dphi = dev_in(h, phi_odd, ce, "stage_in");
  const bool want_force = F != nullptr;  // null: the action only
  const bool staged = want_force && !device_resident(F, h->device);
  double* dF = staged ? h->buf<double>("stage_force", V * 32) : F;
  const char* nm[] = {"fo_phi", "fo_X", "fo_Y", "fo_v1", "fo_v2", "fo_v3", "fo_v4", "fo_v5", "fo_v6",
                      "fo_w1", "fo_w2", "fo_w3", "fo_w4", "fo_w5", "fo_w6"};
  Cx<double>* f[15];
  for (int k = 0; k < 15; ++k) f[k] = h->buf<Cx<double>>(nm[k], n);
  Cx<double>*phi = f[0], *X = f[1], *Y = f[2], *v1 = f[3], *v2 = f[4], *v3 = f[5], *v4 = f[6], *v5 = f[7],
  *v6 = f[8], *w1 = f[9], *w2 = f[10], *w3 = f[11], *w4 = f[12], *w5 = f[13], *w6 = f[14];
  {
    Prof P(h, "import_compact_f64");
    launch_import_compact<double>(g, dphi, phi, 1, 0, frame_rot(h, 1), s);
  }
  // X = (M-hat^dag M-hat)^-1 phi
  int its = precision == WF_FP32 ? cg_normal<float>(h, schur_op<float>(h, 1), schur_op<double>(h, 1), phi, X, n, tol, h->maxiter)
                                 : cg_normal<double>(h, schur_op<double>(h, 1), schur_op<double>(h, 1), phi, X, n, tol, h->maxiter);
  if (iters_out) *iters_out = its;
  // Y = M-hat X and S = phi^dag X = |Y|^2
  double* sc = h->buf<double>("fo_scalars", 2);
  schur_op<double>(h, 1)(X, Y, 0, sc);
  const double S = read_scalars(h, sc, 1)[0];
  if (action) *action = S;
  if (!want_force) return WF_OK;
  const int tp = g.tp;
  auto line = [&](int par, const Cx<double>* in, Cx<double>* out, int opu, int opl) {
    line_load<double>(h, par, in, out, opu, opl, 1, "force_chain_c");
  };
  auto hop = [&](int par_out, const Cx<double>* in, Cx<double>* out, bool adjoint) {
    LineArgs<double> a = line_args<double>(h, par_out, 1);  // D_s^dag = S D_s S (gamma_5-hermiticity)
    a.src_up = in + (adjoint ? 6 * tp : 0);
    a.src_lo = in + (adjoint ? 0 : 6 * tp);
    a.swap_out = adjoint ? 1 : 0;
    a.opu = OP_COPY;
    a.opl = OP_COPY;
    a.src = SRC_HOP;
    a.out = out;
    Prof P(h, "force_chain_hop_f64");
    launch_line<double>(a, LK_GENERIC, h->axial, s);
  };
  // right chain
  line(1, X, v1, OP_FWD, OP_COPY);   // C_R^o
  hop(0, v1, v2, false);             // D^eo
  line(0, v2, v3, OP_COPY, OP_BWD);  // C_L^e
  line(0, v3, v4, OP_FWD, OP_COPY);  // C_R^e
  hop(1, v4, v5, false);             // D^oe
  line(1, v5, v6, OP_COPY, OP_BWD);  // C_L^o
  // left chain (adjoints): C_L^dag = P_+ + P_- T^-dag, C_R^dag = P_- + P_+ T^-1
  line(1, Y, w1, OP_COPY, OP_FWD);
  hop(0, w1, w2, true);
  line(0, w2, w3, OP_BWD, OP_COPY);
  line(0, w3, w4, OP_COPY, OP_FWD);
  hop(1, w4, w5, true);
  line(1, w5, w6, OP_BWD, OP_COPY);
  Gauge<double> G = gauge_of<double>(h);
  for (int p = 0; p < 2; ++p) {
    ForceArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = g;
    a.parity = p;
    a.axial = h->axial;
    a.a = p ? w1 : w4;
    a.b = p ? v6 : v3;
    a.c = p ? w6 : w3;
    a.e = p ? v1 : v4;
    a.w = p ? w1 : w4;
    a.v = p ? v4 : v1;
    a.vr = p ? v1 : v4;
    a.wr = p ? w4 : w1;
    a.ut = G.ut[p];
    a.pl = G.pl[p];
    a.us_p = G.us[p];
    a.coef = 2.0 / (g.gamma_f * g.gamma_f);
    a.bc = g.bc;
    a.F = dF;
    Prof P(h, "force_outer_products_f64", 2);
    launch_force(a, s);
  }
  if (staged) WF_CUDA(cudaMemcpyAsync(F, dF, V * 32 * sizeof(double), cudaMemcpyDeviceToHost, s));
  WF_CUDA(cudaStreamSynchronize(s));
  return WF_OK;
}

template <typename R>
int apply_eo4d_abi(wf_handle* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (nrhs < 1) throw Error(WF_EINVAL, "nrhs must be >= 1");
  if (h->g.T % 2) throw Error(WF_EINVAL, "the 4-D even-odd operator needs an even T");
  const size_t ce = (size_t)nrhs * h->g.L * h->g.L * h->g.L * h->g.T / 2 * NSPIN_C;
  const size_t nt = eo_elems(h) * nrhs;
  const Cx<double>* din = dev_in(h, in_odd, ce, "stage_in");
  bool staged;
  Cx<double>* dout = dev_out(h, out_odd, ce, "stage_out", staged);
  Cx<R>* x = h->buf<Cx<R>>(pname<R>("ap_x"), nt);
  Cx<R>* o = h->buf<Cx<R>>(pname<R>("ap_o"), nt);
  Cx<R>* he = h->buf<Cx<R>>(pname<R>("ap_y"), nt);
  {
    Prof P(h, pname<R>("import_eo"));
    launch_import_eo<R>(h->g, din, nullptr, x, nrhs, frame_rot(h, 0), frame_rot(h, 1), 1, h->stream);
  }
  eo4d_apply<R>(h, x, o, dagger, nrhs, he, nullptr);
  {
    Prof P(h, pname<R>("export_eo"));
    launch_export_eo<R>(h->g, nullptr, o, dout, nrhs, frame_rot(h, 0), frame_rot(h, 1), 1, h->stream);
  }
  finish_out(h, out_odd, dout, ce, staged);
  return WF_OK;
}

template <typename R>
int apply_schur_abi(wf_handle* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (nrhs < 1) throw Error(WF_EINVAL, "nrhs must be >= 1");
  const size_t ce = (size_t)nrhs * h->g.T * h->g.Nl * NSPIN_C;
  const size_t nt = h->half_int() * nrhs;
  const Cx<double>* din = dev_in(h, in_odd, ce, "stage_in");
  bool staged;
  Cx<double>* dout = dev_out(h, out_odd, ce, "stage_out", staged);
  Cx<R>* x = h->buf<Cx<R>>(pname<R>("ap_x"), nt);
  Cx<R>* o = h->buf<Cx<R>>(pname<R>("ap_o"), nt);
  Cx<R>* y = h->buf<Cx<R>>(pname<R>("ap_y"), nt);
  Cx<R>* z = h->buf<Cx<R>>(pname<R>("ap_z"), nt);
  { Prof P(h, pname<R>("import_compact")); launch_import_compact<R>(h->g, din, x, nrhs, 0, frame_rot(h, 1), h->stream); }
  schur_apply<R>(h, x, o, dagger, nrhs, y, z);
  { Prof P(h, pname<R>("export_compact")); launch_export_compact<R>(h->g, o, dout, nrhs, 0, frame_rot(h, 1), h->stream); }
  finish_out(h, out_odd, dout, ce, staged);
  return WF_OK;
}

// M-hat with FP16-stored fields (FP32 arithmetic): the operator of the FP16MIX solve. Each
// source is stored divided by its RMS, so any input range fits FP16.
int apply_schur_f16_abi(wf_handle* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (nrhs < 1) throw Error(WF_EINVAL, "nrhs must be >= 1");
  if (!h->axial || !wide_supported(h->g))
    throw Error(WF_EINVAL, "FP16 storage: the axial frame on lattices the one-thread-per-site kernels serve");
  const size_t n = h->half_int();
  const size_t ce = (size_t)nrhs * h->g.T * h->g.Nl * NSPIN_C;
  const size_t nt = n * nrhs;
  cudaStream_t s = h->stream;
  const Cx<double>* din = dev_in(h, in_odd, ce, "stage_in");
  bool staged;
  Cx<double>* dout = dev_out(h, out_odd, ce, "stage_out", staged);
  Cx<float>* x = h->buf<Cx<float>>(pname<float>("ap_x"), nt);
  Cx<float>* o = h->buf<Cx<float>>(pname<float>("ap_o"), nt);
  Cx16* x16 = h->buf<Cx16>("ap_x16", nt);
  Cx16* o16 = h->buf<Cx16>("ap_o16", nt);
  Cx16* y16 = h->buf<Cx16>("ap_y16", nt);
  Cx16* z16 = h->buf<Cx16>("ap_z16", nt);
  double* sc = h->buf<double>("ap_scale", 2 * (size_t)nrhs);
  double* partial = h->buf<double>("cg_partial", 1024 * (size_t)nrhs);
  { Prof P(h, "import_compact_f32"); launch_import_compact<float>(h->g, din, x, nrhs, 0, frame_rot(h, 1), s); }
  { Prof P(h, "norm2_f32", 2); launch_norm2<float>(x, n, nrhs, partial, sc, s); }
  std::vector<double> x2 = read_scalars(h, sc, nrhs), inv(nrhs), sig(nrhs);
  for (int k = 0; k < nrhs; ++k) {
    sig[k] = x2[k] > 0.0 ? std::sqrt(x2[k] / (double)n) : 1.0;
    inv[k] = 1.0 / sig[k];
  }
  WF_CUDA(cudaMemcpyAsync(sc, inv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(sc + nrhs, sig.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
  { Prof P(h, "h16_scale"); launch_scale_to_h16<Cx<float>>(x16, x, n, nrhs, sc, s); }
  schur_apply_h16(h, x16, o16, dagger, nrhs, y16, z16, nullptr);
  { Prof P(h, "h16_unscale"); launch_scale_from_h16(o, o16, n, nrhs, sc + nrhs, s); }
  { Prof P(h, "export_compact_f32"); launch_export_compact<float>(h->g, o, dout, nrhs, 0, frame_rot(h, 1), s); }
  finish_out(h, out_odd, dout, ce, staged);
  return WF_OK;
}

template <typename R>
int apply_M_abi(wf_handle* h, const double* in, double* out, int dagger, int nrhs) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (nrhs < 1) throw Error(WF_EINVAL, "nrhs must be >= 1");
  const size_t le = h->lex_elems() * nrhs;
  const size_t nt = h->half_int() * nrhs;
  const Cx<double>* din = dev_in(h, in, le, "stage_in");
  bool staged;
  Cx<double>* dout = dev_out(h, out, le, "stage_out", staged);
  Cx<R>* ie = h->buf<Cx<R>>(pname<R>("ap_ie"), nt);
  Cx<R>* io = h->buf<Cx<R>>(pname<R>("ap_io"), nt);
  Cx<R>* oe = h->buf<Cx<R>>(pname<R>("ap_oe"), nt);
  Cx<R>* oo = h->buf<Cx<R>>(pname<R>("ap_oo"), nt);
  { Prof P(h, pname<R>("import_spinor")); launch_import_spinor<R>(h->g, din, ie, io, nrhs, dagger, frame_rot(h, 0), frame_rot(h, 1), h->stream); }
  m_apply<R>(h, ie, io, oe, oo, nullptr, nullptr, 0.0, nrhs);
  { Prof P(h, pname<R>("export_spinor")); launch_export_spinor<R>(h->g, oe, oo, dout, nrhs, dagger, frame_rot(h, 0), frame_rot(h, 1), h->stream); }
  finish_out(h, out, dout, le, staged);
  return WF_OK;
}

template <typename R>
int apply_line_abi(wf_handle* h, const double* in, double* out, int opu, int opl, int nrhs, const char* name) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (nrhs < 1) throw Error(WF_EINVAL, "nrhs must be >= 1");
  const size_t le = h->lex_elems() * nrhs;
  const size_t nt = h->half_int() * nrhs;
  const Cx<double>* din = dev_in(h, in, le, "stage_in");
  bool staged;
  Cx<double>* dout = dev_out(h, out, le, "stage_out", staged);
  Cx<R>* ie = h->buf<Cx<R>>(pname<R>("ap_ie"), nt);
  Cx<R>* io = h->buf<Cx<R>>(pname<R>("ap_io"), nt);
  Cx<R>* oe = h->buf<Cx<R>>(pname<R>("ap_oe"), nt);
  Cx<R>* oo = h->buf<Cx<R>>(pname<R>("ap_oo"), nt);
  { Prof P(h, pname<R>("import_spinor")); launch_import_spinor<R>(h->g, din, ie, io, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), h->stream); }
  line_load<R>(h, 0, ie, oe, opu, opl, nrhs, name);
  line_load<R>(h, 1, io, oo, opu, opl, nrhs, name);
  { Prof P(h, pname<R>("export_spinor")); launch_export_spinor<R>(h->g, oe, oo, dout, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), h->stream); }
  finish_out(h, out, dout, le, staged);
  return WF_OK;
}

// M-tilde_ILU (dagger: gamma_5 M-tilde_ILU gamma_5) on full fields
template <typename R>
int apply_ilu_abi(wf_handle* h, const double* in, double* out, int dagger, int nrhs) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (nrhs < 1) throw Error(WF_EINVAL, "nrhs must be >= 1");
  const size_t le = h->lex_elems() * nrhs;
  const size_t hn = h->half_int(), nt = hn * nrhs;
  const Cx<double>* din = dev_in(h, in, le, "stage_in");
  bool staged;
  Cx<double>* dout = dev_out(h, out, le, "stage_out", staged);
  Cx<R>* ie = h->buf<Cx<R>>(pname<R>("ap_ie"), nt);
  Cx<R>* io = h->buf<Cx<R>>(pname<R>("ap_io"), nt);
  Cx<R>* oe = h->buf<Cx<R>>(pname<R>("ap_oe"), nt);
  Cx<R>* oo = h->buf<Cx<R>>(pname<R>("ap_oo"), nt);
  { Prof P(h, pname<R>("import_spinor")); launch_import_spinor<R>(h->g, din, ie, io, nrhs, dagger, frame_rot(h, 0), frame_rot(h, 1), h->stream); }
  for (int k = 0; k < nrhs; ++k) ilu_apply<R>(h, ie + k * hn, io + k * hn, oe + k * hn, oo + k * hn);
  { Prof P(h, pname<R>("export_spinor")); launch_export_spinor<R>(h->g, oe, oo, dout, nrhs, dagger, frame_rot(h, 0), frame_rot(h, 1), h->stream); }
  finish_out(h, out, dout, le, staged);
  return WF_OK;
}

// out = A in (the clover term alone, site-diagonal) on full fields, FP64
int apply_clover_abi(wf_handle* h, const double* in, double* out, int nrhs) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (!h->clover) throw Error(WF_EINVAL, "no clover term loaded (wf_load_gauge_clover)");
  if (nrhs < 1) throw Error(WF_EINVAL, "nrhs must be >= 1");
  const size_t le = h->lex_elems() * nrhs;
  const size_t nt = h->half_int() * nrhs;
  const Cx<double>* din = dev_in(h, in, le, "stage_in");
  bool staged;
  Cx<double>* dout = dev_out(h, out, le, "stage_out", staged);
  Cx<double>* ie = h->buf<Cx<double>>("ap_ie_f64", nt);
  Cx<double>* io = h->buf<Cx<double>>("ap_io_f64", nt);
  Cx<double>* oe = h->buf<Cx<double>>("ap_oe_f64", nt);
  Cx<double>* oo = h->buf<Cx<double>>("ap_oo_f64", nt);
  { Prof P(h, "import_spinor_f64"); launch_import_spinor<double>(h->g, din, ie, io, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), h->stream); }
  clover_on<double>(h, 0, ie, oe, nullptr, 1.0, nrhs);
  clover_on<double>(h, 1, io, oo, nullptr, 1.0, nrhs);
  { Prof P(h, "export_spinor_f64"); launch_export_spinor<double>(h->g, oe, oo, dout, nrhs, 0, frame_rot(h, 0), frame_rot(h, 1), h->stream); }
  finish_out(h, out, dout, le, staged);
  return WF_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------
extern "C" {

int wf_create(int L, int T, double xi, double kappa_s, double kappa_t, int bc, wf_handle_t** out) {
  if (!out) return WF_EINVAL;
  *out = nullptr;
  if (L < 2 || (L & 1) || T < 2 || T > 256) return WF_EINVAL;
  if (!(kappa_s > 0) || (bc != 1 && bc != -1)) return WF_EINVAL;
  if (!(kappa_t > 0)) {
    if (!(xi > 0)) return WF_EINVAL;
    kappa_t = xi * kappa_s;
  }
  wf_handle* h = nullptr;
  try {
    h = new wf_handle();
    h->xi = xi;
    h->kappa_s = kappa_s;
    h->kappa_t = kappa_t;
    h->g = make_geom(L, T, kappa_s, kappa_t, bc);
    if (const char* e = std::getenv("WF_DF64")) h->df_allowed = e[0] == '1';
    WF_CUDA(cudaGetDevice(&h->device));
    WF_CUDA(cudaMallocHost(&h->host_scalars, 4096 * sizeof(double)));
    *out = h;
    return WF_OK;
  } catch (const Error& e) {
    delete h;
    return e.code;
  } catch (...) {
    delete h;
    return WF_ENOMEM;
  }
}

int wf_destroy(wf_handle_t* h) {
  if (!h) return WF_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& r : h->prof_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->host_scalars) cudaFreeHost(h->host_scalars);
  delete h;
  return WF_OK;
}

int wf_set_stream(wf_handle_t* h, void* stream) {
  return guarded(h, [&]() {
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    return WF_OK;
  });
}

const char* wf_last_error(const wf_handle_t* h) { return h ? h->err.c_str() : "null handle"; }

int wf_set_gauge_frame(wf_handle_t* h, int axial) {
  return guarded(h, [&]() {
    if (axial != 0 && axial != 1) throw Error(WF_EINVAL, "axial must be 0 or 1");
    h->axial = axial != 0;
    h->gauge = false;  // the stored field belongs to the old frame: load the gauge field again
    return WF_OK;
  });
}

long long wf_field_elems(const wf_handle_t* h) { return h ? (long long)h->g.L * h->g.L * h->g.L * h->g.T * 12 : 0; }
long long wf_half_elems(const wf_handle_t* h) { return h ? (long long)h->g.L * h->g.L * h->g.L * h->g.T * 6 : 0; }

int wf_load_gauge(wf_handle_t* h, const double* U) {
  return guarded(h, [&]() {
    h->clover = false;  // a clover term belongs to the field it was built from
    const Geom& g = h->g;
    const size_t V = (size_t)g.L * g.L * g.L * g.T;
    const Cx<double>* dU = dev_in(h, U, V * 36, "stage_gauge");
    {
      int* chk = h->buf<int>("gauge_check", 1);
      WF_CUDA(cudaMemsetAsync(chk, 0, sizeof(int), h->stream));
      launch_check_links(dU, V * 4, 1e-9, chk, h->stream);
      h->launches += 1;
      int bad = 0;
      WF_CUDA(cudaMemcpyAsync(&bad, chk, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      WF_CUDA(cudaStreamSynchronize(h->stream));
      if (bad & 1) throw Error(WF_EINVAL, "gauge field has a NaN or Inf entry");
      if (bad & 2) throw Error(WF_EINVAL, "gauge field has a link that is not SU(3) within 1e-9");
    }
    const size_t nut = (size_t)g.Nl * 9 * g.tp, nus = 3 * nut, nlam = (size_t)g.Nl * 9;
    const size_t nus32 = (size_t)3 * g.Nl * SpatialLinkNC<float>::value * g.tp;
    cudaStream_t s = h->stream;
    for (int p = 0; p < 2; ++p) {
      h->ut64[p].ensure(nut * sizeof(Cx<double>), s);
      h->us64[p].ensure(nus * sizeof(Cx<double>), s);
      h->lamb64[p].ensure(nlam * sizeof(Cx<double>), s);
      h->lamf64[p].ensure(nlam * sizeof(Cx<double>), s);
      if (!h->axial) h->ut32[p].ensure(nut * sizeof(Cx<float>), s);
      h->us32[p].ensure(nus32 * sizeof(Cx<float>), s);
      h->lamb32[p].ensure(nlam * sizeof(Cx<float>), s);
      h->lamf32[p].ensure(nlam * sizeof(Cx<float>), s);
    }
    h->iflag.ensure(sizeof(int), s);
    WF_CUDA(cudaMemsetAsync(h->iflag.p, 0, sizeof(int), s));
    Cx<double>* ut[2] = {h->ut64[0].as<Cx<double>>(), h->ut64[1].as<Cx<double>>()};
    Cx<double>* us[2] = {h->us64[0].as<Cx<double>>(), h->us64[1].as<Cx<double>>()};
    Prof P(h, "gauge_ingest", 1 + 2 * 5);
    launch_import_gauge(g, dU, ut, us, s);
    if (h->axial) {
      // axial frame: ut becomes the rotation g, spatial links rotated in place, P, Lambda and the
      // wrap matrix P Lambda (held in lamf) per line
      for (int p = 0; p < 2; ++p) {
        h->pl64[p].ensure(nlam * sizeof(Cx<double>), s);
        h->pl32[p].ensure(nlam * sizeof(Cx<float>), s);
        launch_axial_frame(g, ut[p], h->pl64[p].as<Cx<double>>(), h->lamb64[p].as<Cx<double>>(),
                           h->lamf64[p].as<Cx<double>>(), h->iflag.as<int>(), s);
      }
      const Cx<double>* gg[2] = {ut[0], ut[1]};
      launch_rotate_links(g, us, gg, s);
      for (int p = 0; p < 2; ++p) {
        launch_d2f_links(us[p], h->us32[p].as<Cx<float>>(), (size_t)3 * g.Nl, g.tp, s);
        launch_d2f(h->pl64[p].as<Cx<double>>(), h->pl32[p].as<Cx<float>>(), nlam, s);
        launch_d2f(h->lamb64[p].as<Cx<double>>(), h->lamb32[p].as<Cx<float>>(), nlam, s);
        launch_d2f(h->lamf64[p].as<Cx<double>>(), h->lamf32[p].as<Cx<float>>(), nlam, s);
      }
    } else {
      for (int p = 0; p < 2; ++p) {
        launch_tline_init(g, ut[p], h->lamb64[p].as<Cx<double>>(), h->lamf64[p].as<Cx<double>>(), h->iflag.as<int>(), s);
        launch_d2f(ut[p], h->ut32[p].as<Cx<float>>(), nut, s);
        launch_d2f_links(us[p], h->us32[p].as<Cx<float>>(), (size_t)3 * g.Nl, g.tp, s);
        launch_d2f(h->lamb64[p].as<Cx<double>>(), h->lamb32[p].as<Cx<float>>(), nlam, s);
        launch_d2f(h->lamf64[p].as<Cx<double>>(), h->lamf32[p].as<Cx<float>>(), nlam, s);
      }
    }
    int flag = 0;
    WF_CUDA(cudaMemcpyAsync(&flag, h->iflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    WF_CUDA(cudaStreamSynchronize(s));
    h->gauge = true;
    if (flag) {
      h->gauge = false;
      throw Error(WF_ESINGULAR, "temporal preconditioner singular: |det(1 - bc mu^-T P)| < 1e-12 on some line");
    }
    return WF_OK;
  });
}

int wf_load_gauge_clover(wf_handle_t* h, const double* U, double c_s, double c_t) {
  const int st = wf_load_gauge(h, U);
  if (st != WF_OK) return st;
  return guarded(h, [&]() {
    if (!std::isfinite(c_s) || !std::isfinite(c_t)) throw Error(WF_EINVAL, "c_s and c_t must be finite");
    const Geom& g = h->g;
    const size_t V = (size_t)g.L * g.L * g.L * g.T;
    cudaStream_t s = h->stream;
    const Cx<double>* dU = dev_in(h, U, V * 36, "stage_gauge");
    const size_t nh = (size_t)g.Nl * 72 * g.tp;
    for (int p = 0; p < 2; ++p) {
      h->clov64[p].ensure(nh * sizeof(Cx<double>), s);
      h->clov32[p].ensure(nh * sizeof(Cx<float>), s);
      WF_CUDA(cudaMemsetAsync(h->clov64[p].p, 0, nh * sizeof(Cx<double>), s));  // padding slots stay zero
    }
    Cx<double>* F = h->buf<Cx<double>>("clover_F", V * 54);
    Cx<double>* H[2] = {h->clov64[0].as<Cx<double>>(), h->clov64[1].as<Cx<double>>()};
    const Cx<double>* rot[2] = {frame_rot(h, 0), frame_rot(h, 1)};
    {
      Prof P(h, "clover_build", 2 + 2);
      launch_clover_build(g, dU, h->axial ? rot : nullptr, c_s, c_t, F, H, s);
      for (int p = 0; p < 2; ++p) launch_d2f(H[p], h->clov32[p].as<Cx<float>>(), nh, s);
    }
    if (g.T % 2 == 0) {  // the 4-D Schur comparator: mu + A and its inverse, 4-D even-odd layout
      const size_t n4 = (size_t)g.L * g.L * g.L * 72 * (g.T / 2);
      for (int p = 0; p < 2; ++p) {
        h->clmu64[p].ensure(n4 * sizeof(Cx<double>), s);
        h->clinv64[p].ensure(n4 * sizeof(Cx<double>), s);
        h->clmu32[p].ensure(n4 * sizeof(Cx<float>), s);
        h->clinv32[p].ensure(n4 * sizeof(Cx<float>), s);
      }
      const Cx<double>* Hc[2] = {H[0], H[1]};
      Cx<double>* M4[2] = {h->clmu64[0].as<Cx<double>>(), h->clmu64[1].as<Cx<double>>()};
      Cx<double>* Mi4[2] = {h->clinv64[0].as<Cx<double>>(), h->clinv64[1].as<Cx<double>>()};
      WF_CUDA(cudaMemsetAsync(h->iflag.p, 0, sizeof(int), s));
      Prof P(h, "clover_eo4_build", 1 + 4);
      launch_clover_eo4_build(g, Hc, M4, Mi4, h->iflag.as<int>(), s);
      for (int p = 0; p < 2; ++p) {
        launch_d2f(M4[p], h->clmu32[p].as<Cx<float>>(), n4, s);
        launch_d2f(Mi4[p], h->clinv32[p].as<Cx<float>>(), n4, s);
      }
      int flag = 0;
      WF_CUDA(cudaMemcpyAsync(&flag, h->iflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      WF_CUDA(cudaStreamSynchronize(s));
      if (flag) throw Error(WF_ESINGULAR, "mu + A is singular on some site");
    }
    WF_CUDA(cudaStreamSynchronize(s));
    h->ws.erase("clover_F");  // V x 6 field-strength matrices: needed only while building
    h->c_s = c_s;
    h->c_t = c_t;
    h->clover = true;
    return WF_OK;
  });
}

int wf_apply_clover(wf_handle_t* h, const double* in, double* out, int nrhs) {
  return guarded(h, [&]() { return apply_clover_abi(h, in, out, nrhs); });
}
int wf_apply_ilu(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs) {
  return guarded(h, [&]() { return apply_ilu_abi<double>(h, in, out, dagger ? 1 : 0, nrhs); });
}
int wf_apply_ilu_f32(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs) {
  return guarded(h, [&]() { return apply_ilu_abi<float>(h, in, out, dagger ? 1 : 0, nrhs); });
}

int wf_apply_M(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs) {
  return guarded(h, [&]() { return apply_M_abi<double>(h, in, out, dagger ? 1 : 0, nrhs); });
}
int wf_apply_M_f32(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs) {
  return guarded(h, [&]() { return apply_M_abi<float>(h, in, out, dagger ? 1 : 0, nrhs); });
}
int wf_apply_Tinv(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs) {
  return guarded(h, [&]() {
    int op = dagger ? OP_FWD : OP_BWD;
    return apply_line_abi<double>(h, in, out, op, op, nrhs, "tinv");
  });
}
int wf_apply_Tinv_f32(wf_handle_t* h, const double* in, double* out, int dagger, int nrhs) {
  return guarded(h, [&]() {
    int op = dagger ? OP_FWD : OP_BWD;
    return apply_line_abi<float>(h, in, out, op, op, nrhs, "tinv");
  });
}
int wf_apply_C(wf_handle_t* h, const double* in, double* out, int which, int nrhs) {
  return guarded(h, [&]() {
    if (which == 0) return apply_line_abi<double>(h, in, out, OP_COPY, OP_BWD, nrhs, "c_left");
    if (which == 1) return apply_line_abi<double>(h, in, out, OP_FWD, OP_COPY, nrhs, "c_right");
    throw Error(WF_EINVAL, "which must be 0 (C_L) or 1 (C_R)");
  });
}
int wf_apply_schur(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  return guarded(h, [&]() { return apply_schur_abi<double>(h, in_odd, out_odd, dagger ? 1 : 0, nrhs); });
}
int wf_apply_schur_f32(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  return guarded(h, [&]() { return apply_schur_abi<float>(h, in_odd, out_odd, dagger ? 1 : 0, nrhs); });
}

int wf_apply_schur_f16(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  return guarded(h, [&]() { return apply_schur_f16_abi(h, in_odd, out_odd, dagger ? 1 : 0, nrhs); });
}

int wf_force(wf_handle_t* h, const double* phi_odd, double* F, int precision, double tol, double* action,
             int* iters) {
  return guarded(h, [&]() {
    if (precision != WF_FP64 && precision != WF_FP32) throw Error(WF_EINVAL, "unknown precision");
    return force_abi(h, phi_odd, F, precision, tol, action, iters);
  });
}

int wf_apply_eo4d(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  return guarded(h, [&]() { return apply_eo4d_abi<double>(h, in_odd, out_odd, dagger ? 1 : 0, nrhs); });
}
int wf_apply_eo4d_f32(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  return guarded(h, [&]() { return apply_eo4d_abi<float>(h, in_odd, out_odd, dagger ? 1 : 0, nrhs); });
}

int wf_solve(wf_handle_t* h, const double* rhs, double* x, int nrhs, double tol, int method, int precision, int flags,
             int* iters_out, double* true_resid_out) {
  return guarded(h, [&]() {
    if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
    if (nrhs < 1 || nrhs > WF_MAX_SOLVE_RHS) throw Error(WF_EINVAL, "nrhs must lie in [1, WF_MAX_SOLVE_RHS]");
    if (!(tol > 0)) throw Error(WF_EINVAL, "tol must be > 0");
    if (precision != WF_FP64 && precision != WF_FP32 && precision != WF_FP16MIX)
      throw Error(WF_EINVAL, "unknown precision");
    if (precision == WF_FP16MIX && (method != WF_TEMPORAL_SCHUR || !h->axial || !wide_supported(h->g)))
      throw Error(WF_EINVAL, "WF_FP16MIX: the temporal + Schur method in the axial frame on lattices whose time lines "
                             "the one-thread-per-site kernels serve");
    const size_t le = h->lex_elems() * nrhs;
    const bool x0 = (flags & WF_X0) != 0;
    const Cx<double>* drhs = dev_in(h, rhs, le, "stage_in");
    bool staged;
    Cx<double>* dx = dev_out(h, x, le, "stage_out", staged);
    if (x0 && staged) WF_CUDA(cudaMemcpyAsync(dx, x, le * sizeof(Cx<double>), cudaMemcpyHostToDevice, h->stream));
    if (h->clover && method != WF_TEMPORAL_ILU && method != WF_EO4D)
      throw Error(WF_EINVAL, "a clover term is loaded: WF_TEMPORAL_ILU and WF_EO4D are the methods that solve M + A");
    if (method == WF_TEMPORAL_ILU && x0) throw Error(WF_EINVAL, "WF_TEMPORAL_ILU takes no initial guess");
    int st;
    if (method == WF_TEMPORAL_ILU)
      st = solve_temporal_ilu(h, drhs, dx, nrhs, tol, precision, iters_out, true_resid_out);
    else if (method == WF_TEMPORAL_SCHUR)
      st = solve_temporal_schur(h, drhs, dx, nrhs, tol, precision, x0, iters_out, true_resid_out);
    else if (method == WF_EO4D)
      st = solve_eo4d(h, drhs, dx, nrhs, tol, precision, x0, iters_out, true_resid_out);
    else if (method == WF_UNPREC || method == WF_TEMPORAL)
      st = solve_full(h, drhs, dx, nrhs, tol, precision, x0, method == WF_TEMPORAL, iters_out, true_resid_out);
    else
      throw Error(WF_EINVAL, "unknown method");
    finish_out(h, x, dx, le, staged);
    if (st == WF_ENOCONV) h->err = "solver did not reach tol";
    return st;
  });
}

int wf_solve_many(int n, wf_handle_t* const* hs, const double* const* rhs, double* const* x, const int* nrhs,
                  double tol, int method, int precision, int flags, int* const* iters_out,
                  double* const* resid_out, int* status_out) {
  if (n < 1 || !hs || !rhs || !x || !nrhs) return WF_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return WF_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return WF_EINVAL;  // one handle per lattice: a handle is not shared
  }
  std::vector<int> st(n, WF_OK);
  if (joint_eligible(n, hs, method, precision) && joint_fits(n, nrhs)) {
    solve_many_joint(n, hs, rhs, x, nrhs, tol, flags, iters_out, resid_out, st);
    int first = WF_OK;
    for (int i = 0; i < n; ++i) {
      if (status_out) status_out[i] = st[i];
      if (first == WF_OK && st[i] != WF_OK) first = st[i];
    }
    return first;
  }
  std::vector<cudaStream_t> own(n, nullptr);
  try {
    // every solve on a stream of its own (a temporary one for handles on the default stream)
    for (int i = 0; i < n; ++i) {
      if (hs[i]->stream) continue;
      int prev = 0;
      if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(hs[i]->device) != cudaSuccess) throw Error(WF_ECUDA, "device");
      const cudaError_t e = cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking);
      cudaSetDevice(prev);
      if (e != cudaSuccess) throw Error(WF_ECUDA, "cudaStreamCreateWithFlags");
      hs[i]->stream = own[i];
    }
    std::vector<std::thread> th;
    th.reserve(n);
    for (int i = 0; i < n; ++i)
      th.emplace_back([&, i]() {
        if (cudaSetDevice(hs[i]->device) != cudaSuccess) {
          st[i] = WF_ECUDA;
          return;
        }
        st[i] = wf_solve(hs[i], rhs[i], x[i], nrhs[i], tol, method, precision, flags,
                         iters_out ? iters_out[i] : nullptr, resid_out ? resid_out[i] : nullptr);
      });
    for (auto& t : th) t.join();
  } catch (const Error& e) {
    for (int i = 0; i < n; ++i)
      if (st[i] == WF_OK) st[i] = e.code;
  } catch (...) {
    for (int i = 0; i < n; ++i)
      if (st[i] == WF_OK) st[i] = WF_ENOMEM;
  }
  for (int i = 0; i < n; ++i) {
    if (!own[i]) continue;
    cudaStreamSynchronize(own[i]);
    hs[i]->stream = nullptr;
    cudaStreamDestroy(own[i]);
  }
  int first = WF_OK;
  for (int i = 0; i < n; ++i) {
    if (status_out) status_out[i] = st[i];
    if (first == WF_OK && st[i] != WF_OK) first = st[i];
  }
  return first;
}

int wf_hop_config(wf_handle_t* h, int nrhs, int* variant, int* tile_rows, float* ms) {
  return guarded(h, [&]() {
    auto it = h->hop_tune.find(nrhs);
    if (it == h->hop_tune.end()) throw Error(WF_EINVAL, "no tuned hop configuration for this nrhs yet");
    if (variant) *variant = it->second.variant;
    if (tile_rows) *tile_rows = it->second.by;
    if (ms) *ms = it->second.ms;
    return WF_OK;
  });
}

int wf_hop_pipe_config(wf_handle_t* h, int nrhs, int* sources_per_unit, int* stages) {
  return guarded(h, [&]() {
    auto it = h->hop_tune.find(nrhs);
    if (it == h->hop_tune.end()) throw Error(WF_EINVAL, "no tuned hop configuration for this nrhs yet");
    const bool pipe = it->second.variant == 3;
    if (sources_per_unit) *sources_per_unit = pipe ? it->second.gsrc : 0;
    if (stages) *stages = pipe ? it->second.ns : 0;
    return WF_OK;
  });
}

int wf_set_max_iterations(wf_handle_t* h, int maxiter) {
  return guarded(h, [&]() {
    if (maxiter < 0) throw Error(WF_EINVAL, "maxiter must be >= 0");
    h->maxiter = maxiter ? maxiter : 100000;
    return WF_OK;
  });
}

long long wf_launch_count(const wf_handle_t* h) { return h ? h->launches : 0; }

int wf_check_tables(int L, int T, int nrhs, int tile_rows, int plant) {
  try {
    if (nrhs < 1 || nrhs > WF_MAX_SOLVE_RHS || plant < 0 || plant > 3) return WF_EINVAL;
    Geom g = make_geom(L, T, 0.1, 0.3, -1);
    if (tile_rows > 0) {
      if (tile_rows > L || L % tile_rows) return WF_EINVAL;
      g.by = tile_rows;
    }
    for (int p = 0; p < 2; ++p) {
      std::vector<int> t = build_nbr_table(g, p);
      if (plant == 1 && p == 1) {
        std::swap(t[0], t[t.size() - 1]);  // two lines' neighbours exchanged
        check_nbr_table(g, p, t);
      }
    }
    std::vector<int2> o = build_order_table(g, nrhs);
    if (plant == 2) {
      o[o.size() / 2] = o[0];  // one pair visited twice, another never
      check_order_table(g, nrhs, o);
    }
    for (int gs = 1; gs <= 2; ++gs) {
      std::vector<int2> u = build_unit_table(g, nrhs, gs);
      if (plant == 3 && gs == 2) {
        u.back().y = g.Nl;  // a line past the end
        check_unit_table(g, nrhs, gs, u);
      }
    }
    return WF_OK;
  } catch (const Error& e) {
    return e.code;
  } catch (...) {
    return WF_ENOMEM;
  }
}

int wf_profile(wf_handle_t* h, int on) {
  return guarded(h, [&]() {
    h->fold_pending();
    if (on) {
      std::fill(h->prof_count.begin(), h->prof_count.end(), 0);
      std::fill(h->prof_ms.begin(), h->prof_ms.end(), 0.0);
    }
    h->prof = on != 0;
    return WF_OK;
  });
}

int wf_profile_get(wf_handle_t* h, const char** names, long long* launches, double* total_ms, int cap) {
  if (!h) return -WF_EINVAL;
  try {
    h->fold_pending();
  } catch (const Error& e) {
    h->err = e.what();
    return -e.code;
  }
  int n = (int)h->prof_names.size();
  for (int i = 0; i < n && i < cap; ++i) {
    if (names) names[i] = h->prof_names[i].c_str();
    if (launches) launches[i] = h->prof_count[i];
    if (total_ms) total_ms[i] = h->prof_ms[i];
  }
  return n;
}

}  // extern "C"
