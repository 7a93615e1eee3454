// graf_noalloc.cu - graf_af_loss_backward for callers that cannot allocate
// device memory.
//
// Some callers cannot hand this library a workspace: a radar processing loop
// that fixes its memory map at start-up and treats any later allocation as a
// fault, a host framework whose own pool owns every byte of device memory and
// exposes no allocator to plug-ins, or code on a latency budget that cannot
// afford cudaMalloc's implicit device synchronisation.  For them this file
// keeps the workspace in a fixed device array that the module holds for as
// long as the library is loaded, on every GPU that loads it.
//
// The array is reached from host code only through cudaGetSymbolAddress: on
// the host, the name `g_noalloc_scratch` is a stand-in object, not a device
// address, and must never be passed to a kernel.  The address is looked up on
// every call, in the context current at that call: a device reset or a
// caller-created (non-primary) context gives the array a new address, so no
// address is kept from one call to the next.
#include <cuda_runtime.h>

#include "graf.h"

namespace {

// GRAF_NOALLOC_SCRATCH_BYTES of device memory, 256-byte aligned.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GRAF_NOALLOC_SCRATCH_BYTES];

}  // namespace

extern "C" graf_status_t graf_af_loss_backward_noalloc(const void* x, graf_input_t kind, int32_t B,
                                                        int32_t N, int32_t M, graf_window_t w,
                                                        graf_loss_t l, float* out8, const float* dL,
                                                        graf_c32* grad_s, float* grad_phi,
                                                        void* stream) {
    const size_t need = graf_af_backward_workspace_bytes(B, N, M, w);
    if (need == 0) return GRAF_ERR_INVALID_ARG;
    if (need > (size_t)GRAF_NOALLOC_SCRATCH_BYTES) return GRAF_ERR_WORKSPACE;
    // the array's address in the current context (the first call in a context
    // loads the module there)
    void* scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch) return GRAF_ERR_CUDA;
    // every scratch byte the kernels read is written earlier in the same call
    // (per-CTA records and partial gradients), so nothing needs clearing
    return graf_af_loss_backward(x, kind, B, N, M, w, l, out8, dL, grad_s, grad_phi, scratch,
                                 (size_t)GRAF_NOALLOC_SCRATCH_BYTES, stream);
}
