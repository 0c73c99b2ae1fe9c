// Allocation-free variant of the shearlet analysis.
//
// Some callers cannot allocate device memory at the moment they need a
// transform: code running inside a real-time loop that must not stall on the
// allocator, plugins whose host application owns every device allocation,
// or tools that forbid cudaMalloc after start-up.  shearlet_analyze takes its
// temporaries from the stream-ordered pool; shearlet_analyze_noalloc instead
// uses one fixed scratch array that is part of the library image.  The array
// is reserved on every GPU that loads the library and stays reserved until the
// process exits.
#include <mutex>
#include <string>

#include "shearseg.h"
#include "shf_internal.h"

namespace {

// Scratch for one call: the row spectra of the input channels followed by the
// coefficient spectra, nch * (eta + 1) * H * (W/2 + 1) complex values.
constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};  // device address of g_scratch, per device

// Device address of the scratch array on device `dev`, which must be the
// current device.  The name g_scratch in host code is only a host-side
// stand-in, so the address is looked up once per device with that device
// current.
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return shf::set_error(SHF_ERR_CUDA, "device ordinal out of range");
  cudaError_t e = cudaSuccess;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return shf::set_error(SHF_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return SHF_OK;
}

}  // namespace

extern "C" {

int shearlet_analyze_noalloc(const shf_bank* bank, const float* u, int nch, float* coef, void* stream) {
  if (!bank || !u || !coef || nch < 1)
    return shf::set_error(SHF_ERR_ARG, "shearlet_analyze_noalloc: NULL pointer or nch < 1");
  if ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(coef)) & 7u)
    return shf::set_error(SHF_ERR_ARG, "shearlet_analyze_noalloc: u and coef must be 8-byte aligned");
  shf::Geo g;
  shf::bank_geo(bank, &g);  // the same device tables shearlet_analyze uses
  const int H = g.H, W = g.W, eta = g.eta;
  const size_t ph = static_cast<size_t>(H) * g.Wh;
  const size_t need = sizeof(float2) * ph * static_cast<size_t>(nch) * (1 + static_cast<size_t>(eta));
  if (need > kScratchBytes)
    return shf::set_error(SHF_ERR_SIZE, "shearlet_analyze_noalloc: needs " + std::to_string(need) +
                                            " bytes of scratch (nch * (eta + 1) * H * (W/2 + 1) * 8), more than the "
                                            "fixed " + std::to_string(kScratchBytes) + " bytes");
  // The bank's tables and the scratch must belong to the same GPU: the
  // scratch address is that of the current device.
  int dev = 0;
  cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess)
    return shf::set_error(SHF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ed));
  if (dev != shf::bank_device(bank))
    return shf::set_error(SHF_ERR_STATE, "shearlet_analyze_noalloc: the current device (" + std::to_string(dev) +
                                             ") is not the device the bank was built on (" +
                                             std::to_string(shf::bank_device(bank)) + ")");
  void* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float2* Ur = static_cast<float2*>(base);
  float2* Y = Ur + ph * nch;
  // Every scratch element read below is first written by this call, so nothing
  // has to be cleared between calls.
  cudaError_t e = shf::run_row_r2c(g, u, Ur, nch, 1.f, st);
  if (e == cudaSuccess) e = shf::run_col_fan(g, Ur, Y, nch, shf::default_groups(g, nch), st);
  if (e == cudaSuccess) e = shf::run_row_c2r(g, Y, coef, nch * eta, 1.f / (static_cast<float>(H) * W), st);
  if (e != cudaSuccess)
    return shf::set_error(SHF_ERR_CUDA, std::string("shearlet_analyze_noalloc: ") + cudaGetErrorString(e));
  return SHF_OK;
}

}  // extern "C"
