// Allocation-free entry point for 3D FOF: callers that cannot allocate device memory get
// the same labels as vr_fof3d, with the scratch taken from one static device array of
// fixed size instead of a caller workspace. This adds a second route into the existing
// FOF kernels; the kernels themselves are unchanged.
#include "vr_internal.cuh"
#include "vr_workspace.h"

namespace {

// Scratch shared by every call on a device (held by the device until the process exits).
static __device__ __align__(256) unsigned char g_fof3d_scratch[VR_FOF3D_NOALLOC_BYTES];

// Device address of the static array in the current context. It is looked up on every
// call (no allocation, no synchronisation): a cached address would go stale if the
// context were destroyed and created again (cudaDeviceReset reloads the module). In host
// code the array's name is only a stand-in, so the kernels must be given this address,
// never the symbol itself.
cudaError_t scratch_address(void **out) { return cudaGetSymbolAddress(out, g_fof3d_scratch); }

}  // namespace

extern "C" vr_status vr_fof3d_noalloc(const int32_t *pos, int64_t n, int64_t link_d2,
                                      int32_t *label, void *stream) {
  if (n < 0 || n > VR_FOF3D_NOALLOC_MAX_N) return VR_ERR_INVALID_ARG;
  if (n == 0) return VR_OK;
  if (!pos || !label) return VR_ERR_INVALID_ARG;
  if (vr::ws_fof3d(n) > (size_t)VR_FOF3D_NOALLOC_BYTES) return VR_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VR_ERR_CUDA;
  void *scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return VR_ERR_CUDA;
  // A context on the stack: vr_fof3d uses it only for its error text and event timers
  // (off), so nothing is allocated here.
  vr_ctx local;
  memset(&local, 0, sizeof(local));
  local.device = dev;
  return vr_fof3d(&local, pos, n, link_d2, label, scratch, (size_t)VR_FOF3D_NOALLOC_BYTES, stream);
}
