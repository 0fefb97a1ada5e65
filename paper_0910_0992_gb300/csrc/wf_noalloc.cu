// wf_apply_schur_noalloc: the M-hat apply of wf_apply_schur (FP64) with all of its work
// memory in one fixed device array that the library reserves for itself, so the call
// itself allocates nothing.
//
// Who needs it: callers that cannot let a library call cudaMalloc at apply time, for
// example applications whose own pool allocator has reserved nearly all device memory
// up front (an extra cudaMalloc would fail or fragment the pool), latency-critical loops
// (cudaFree synchronises the whole device, and a growing work buffer would stall the
// first call at a new size), or processes with a device-memory budget fixed at start-up.
//
// Contract (also in include/wf.h):
// * The work memory is the file-scope array below, WF_NOALLOC_SCRATCH_BYTES = 16 MiB per
//   device. It exists on every GPU on which this code is loaded and stays there until the
//   process exits.
// * Host code cannot use the array's name as a device pointer, so every call looks up its
//   device address with cudaGetSymbolAddress, with the handle's device current. The address
//   belongs to the current CUDA context; looking it up per call keeps it valid after a
//   cudaDeviceReset or under another context on the same device.
// * Every call on a device uses the same array and leaves its contents behind; each call
//   clears the part it uses before use. Calls whose device work overlaps (other streams,
//   other handles, other host threads) race on the array: order them.
// * The call returns after its work has finished (it synchronises the handle's stream).
// * in_odd and out_odd must be device memory of the handle's GPU; sizes beyond the array
//   are rejected.
#include <cstring>
#include <string>

#include "wf_handle.h"
#include "wf_line.cuh"

using namespace wf;

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of the array in the current context
void* scratch_address() {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) throw Error(WF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  return p;
}

int noalloc_apply(wf_handle* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  if (!h->gauge) throw Error(WF_EINVAL, "no gauge field loaded");
  if (nrhs < 1) throw Error(WF_EINVAL, "nrhs must be >= 1");
  if (!in_odd || !out_odd || !device_resident(in_odd, h->device) || !device_resident(out_odd, h->device))
    throw Error(WF_EINVAL, "wf_apply_schur_noalloc needs device pointers (host staging would allocate)");
  const size_t nt = h->half_int() * (size_t)nrhs;
  const size_t field_bytes = ((nt * sizeof(Cx<double>) + 255) / 256) * 256;
  const size_t need = 4 * field_bytes;
  if (need > kScratchBytes)
    throw Error(WF_EINVAL, "wf_apply_schur_noalloc: this lattice and nrhs need " + std::to_string(need) +
                               " bytes of work memory; the fixed maximum is " + std::to_string(kScratchBytes));
  unsigned char* base = static_cast<unsigned char*>(scratch_address());
  auto* x = reinterpret_cast<Cx<double>*>(base);
  auto* o = reinterpret_cast<Cx<double>*>(base + field_bytes);
  auto* y = reinterpret_cast<Cx<double>*>(base + 2 * field_bytes);
  auto* z = reinterpret_cast<Cx<double>*>(base + 3 * field_bytes);
  cudaStream_t s = h->stream;
  // the array keeps the previous call's data: padding slots of the fields must start at zero
  WF_CUDA(cudaMemsetAsync(base, 0, need, s));
  const bool prof = h->prof;
  h->prof = false;  // no event creation on this path
  try {
    launch_import_compact<double>(h->g, reinterpret_cast<const Cx<double>*>(in_odd), x, nrhs, 0, frame_rot(h, 1), s);
    h->launches += 1;
    schur_apply<double>(h, x, o, dagger ? 1 : 0, nrhs, y, z);
    launch_export_compact<double>(h->g, o, reinterpret_cast<Cx<double>*>(out_odd), nrhs, 0, frame_rot(h, 1), s);
    h->launches += 1;
  } catch (...) {
    h->prof = prof;
    throw;
  }
  h->prof = prof;
  WF_CUDA(cudaStreamSynchronize(s));
  return WF_OK;
}

}  // namespace

extern "C" int wf_apply_schur_noalloc(wf_handle_t* h, const double* in_odd, double* out_odd, int dagger, int nrhs) {
  if (!h) return WF_EINVAL;
  h->err.clear();
  try {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) WF_CUDA(cudaSetDevice(h->device));
    return noalloc_apply(h, in_odd, out_odd, dagger, nrhs);
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
