// graf_optim.cu - on-device optimiser for phase codes: Adam (the optimiser of
// the paper's experiments, Sec. 7.1.2, learning rate 0.01) with the step count
// held on the device, so a captured CUDA graph of many steps replays without
// any host involvement, and a loss-history recorder.
#include <cuda_runtime.h>
#include <math.h>

#include "graf.h"

namespace graf {
int device_sm_count();  // graf_af.cu
}

namespace {

// One Adam update (Kingma & Ba): t = *step + 1,
//   m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,
//   x -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
// The last block to finish increments *step (every block has read it by then).
__global__ void adam_kernel(float* __restrict__ x, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long long count, graf_adam_t hp,
                            int32_t* step, unsigned int* done) {
    const int t = *step + 1;
    const float c1 = 1.0f / (1.0f - powf(hp.beta1, (float)t));
    const float c2 = 1.0f / (1.0f - powf(hp.beta2, (float)t));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(hp.beta1, m[i], (1.0f - hp.beta1) * gi);
        const float vi = fmaf(hp.beta2, v[i], (1.0f - hp.beta2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        x[i] -= hp.lr * (mi * c1) / (sqrtf(vi * c2) + hp.eps);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(done, 1u);
        if (prev == gridDim.x - 1) {
            *step = t;
            *done = 0u;
            __threadfence();
        }
    }
}

__global__ void record_loss_kernel(const float* __restrict__ out8, int32_t B, float* __restrict__ history,
                                   int32_t history_len, const int32_t* step) {
    const int t = *step;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B && t >= 0 && t < history_len) history[(size_t)t * B + b] = out8[(size_t)b * 8];
}

}  // namespace

extern "C" {

size_t graf_adam_state_bytes(void) { return 256; }

graf_status_t graf_adam_step(float* x, float* m, float* v, const float* grad, int64_t count,
                             graf_adam_t hp, int32_t* step, void* state, void* stream) {
    if (!x || !m || !v || !grad || !step || !state || count < 1) return GRAF_ERR_INVALID_ARG;
    if (!(hp.lr > 0.0f) || !(hp.beta1 >= 0.0f && hp.beta1 < 1.0f) || !(hp.beta2 >= 0.0f && hp.beta2 < 1.0f) ||
        !(hp.eps > 0.0f))
        return GRAF_ERR_INVALID_ARG;
    long long blocks = (count + 255) / 256;
    const long long cap = 4LL * graf::device_sm_count();
    if (blocks > cap) blocks = cap;
    adam_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        x, m, v, grad, count, hp, step, static_cast<unsigned int*>(state));
    return cudaGetLastError() == cudaSuccess ? GRAF_OK : GRAF_ERR_CUDA;
}

graf_status_t graf_record_loss(const float* out8, int32_t B, float* history, int32_t history_len,
                               const int32_t* step, void* stream) {
    if (!out8 || !history || !step || B < 1 || history_len < 1) return GRAF_ERR_INVALID_ARG;
    record_loss_kernel<<<(B + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(out8, B, history,
                                                                                       history_len, step);
    return cudaGetLastError() == cudaSuccess ? GRAF_OK : GRAF_ERR_CUDA;
}

}  // extern "C"
