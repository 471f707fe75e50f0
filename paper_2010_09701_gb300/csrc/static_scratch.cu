// Y = (M^O)^{-1} H^O X without any device allocation, for callers that cannot
// call cudaMalloc (see oefe_apply_a_noalloc in include/oefe.h).
//
// The per-cell products and the enrichment-row sums that oefe_apply_a keeps in
// its growable workspace live here in one file-scope device array of fixed
// size instead. Host code only sees a stand-in symbol for that array, so its
// device address is looked up once per device with cudaGetSymbolAddress while
// that device is current, and the address is what the kernels receive.
#include <cstdint>
#include <mutex>

#include "oefe_internal.h"

namespace {

// Resident on every device that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[OEFE_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_scratch_addr[MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

int scratch_address(oefe_ctx* c, void** out) {
  if (c->device < 0 || c->device >= MAX_DEVICES) {
    c->err = "apply_a_noalloc: device index out of range";
    return OEFE_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[c->device]) {
    // the context's device is current here (every entry point selects it first)
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      c->err = std::string("apply_a_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return OEFE_ERR_CUDA;
    }
    g_scratch_addr[c->device] = p;
  }
  *out = g_scratch_addr[c->device];
  return OEFE_OK;
}

}  // namespace

int apply_a_noalloc(oefe_ctx* c, int ik, const void* X, void* Y, int nv, int ld, int dtype) {
  void* scratch = nullptr;
  OEFE_TRY(scratch_address(c, &scratch));
  return apply_op_scratch(c, ik, X, ld, Y, ld, nv, dtype, true, scratch, (size_t)OEFE_NOALLOC_SCRATCH_BYTES);
}
