// Right-hand sides without any device allocation: smr_rhs_plane_waves_static.
//
// smr_rhs_plane_waves computes, per shape and plane wave, the surface sums
// <psi_n, E_inc> / <psi_n, H_inc> about the particle centre into a scratch
// buffer it allocates with cudaMallocAsync, then multiplies them by each
// particle's phase.  This file provides the same computation with that
// scratch held in a fixed array in device global memory, declared below, so
// the call itself never allocates or frees.
#include <mutex>

#include "smr_internal.h"

namespace {

// Scratch of the shape sums, [S][n_psi][2][R] complex128.  4 MiB on every GPU
// that loads the library, held until the process exits.
constexpr size_t kScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_rhs_scratch[kScratchBytes];

// Device address of g_rhs_scratch per device ordinal, looked up once per
// device with that device current (host code only sees a host-side stand-in
// under the symbol's name, never a usable device address).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(smr::Ctx* c, void** out) {
  if (c->device < 0 || c->device >= kMaxDevices) {
    c->err = "device ordinal out of range for the static scratch table";
    return SMR_E_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[c->device]) {
    int cur = -1;
    SMR_CUDA(c, cudaGetDevice(&cur));
    SMR_CUDA(c, cudaSetDevice(c->device));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (cur >= 0) cudaSetDevice(cur);
    if (e != cudaSuccess || !p) {
      c->err = std::string("cudaGetSymbolAddress(g_rhs_scratch): ") + cudaGetErrorString(e);
      return SMR_E_CUDA;
    }
    g_addr[c->device] = p;
  }
  *out = g_addr[c->device];
  return SMR_OK;
}

}  // namespace

extern "C" int smr_rhs_plane_waves_static(smr_ctx* h, int R, const double* khat, const double* pol,
                                          void* b, void* stream) {
  if (!h || R <= 0 || !khat || !pol || !b) return SMR_E_INVALID_ARG;
  smr::Ctx* c = &h->c;
  if (!c->have_scene) {
    c->err = "no scene: call smr_set_scene first";
    return SMR_E_STATE;
  }
  size_t need = (size_t)c->S * c->npsi * 2 * (size_t)R * sizeof(double2);
  if (need > kScratchBytes) {
    c->err = "smr_rhs_plane_waves_static: shapes x n_psi x 2 x R x 16 bytes = " + std::to_string(need) +
             " exceeds the fixed scratch of " + std::to_string(kScratchBytes) +
             " bytes; use fewer right-hand sides per call";
    return SMR_E_INVALID_ARG;
  }
  void* scratch = nullptr;
  int rc = scratch_address(c, &scratch);
  if (rc) return rc;
  // the kernels, the scene tables and the scratch address all belong to the
  // context's device; like the other entry points, the call leaves it current
  SMR_CUDA(c, cudaSetDevice(c->device));
  // every element of the scratch that is read is written first by the shape
  // kernel of this call, so nothing needs clearing
  return smr::launch_rhs_scratch(c, R, khat, (const double2*)pol, (double2*)scratch, (double2*)b,
                                 (cudaStream_t)stream);
}
