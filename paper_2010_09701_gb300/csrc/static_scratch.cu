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
struct ScratchAddr {
  void* addr = nullptr;   // device address of g_noalloc_scratch
  void* owner = nullptr;  // the CUDA context that address belongs to
};
ScratchAddr g_scratch_addr[MAX_DEVICES];
std::mutex g_scratch_mutex;

// The CUDA context current on this thread (driver entry point, no link-time dependency on libcuda),
// or null when it cannot be queried. A device reset replaces the primary context, and with it the
// module that holds the array, so an address is only reused while its context is still current.
void* current_context() {
  typedef int (*ctx_get_current_fn)(void**);
  static ctx_get_current_fn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (ctx_get_current_fn)p;
    cudaGetLastError();
  }
  void* cur = nullptr;
  if (!fn || fn(&cur) != 0) return nullptr;
  return cur;
}

int scratch_address(oefe_ctx* c, void** out) {
  if (c->device < 0 || c->device >= MAX_DEVICES) {
    c->err = "apply_a_noalloc: device index out of range";
    return OEFE_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchAddr& s = g_scratch_addr[c->device];
  void* cur = current_context();
  if (!s.addr || !cur || cur != s.owner) {
    // the context's device is current here (every entry point selects it first); the lookup is
    // repeated whenever the current context is not the one the cached address came from
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      c->err = std::string("apply_a_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return OEFE_ERR_CUDA;
    }
    s.addr = p;
    s.owner = cur;
  }
  *out = s.addr;
  return OEFE_OK;
}

}  // namespace

int apply_a_noalloc(oefe_ctx* c, int ik, const void* X, void* Y, int nv, int ld, int dtype) {
  void* scratch = nullptr;
  OEFE_TRY(scratch_address(c, &scratch));
  return apply_op_scratch(c, ik, X, ld, Y, ld, nv, dtype, true, scratch, (size_t)OEFE_NOALLOC_SCRATCH_BYTES);
}
