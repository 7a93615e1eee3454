// graf_mlp.cu - the learned proposal network: an MLP that maps a design spec
// to initial phase codes (the "neural network -> waveform -> GRAF layer ->
// loss" pipeline of the paper's Sec. 6.1), trained and run entirely by these
// kernels.  BF16 operands on the 5th-generation tensor cores (tcgen05.mma,
// accumulators in tensor memory), FP32 accumulation, FP32 master weights.
//
// Layer l: Y = X W_l + b_l (X [rows][K] bf16 row-major, W_l [K][N] bf16
// row-major, b_l fp32), followed by GELU on the hidden layers.  Activations
// are stored in bf16 (the next GEMM's operand) and the pre-activations in
// fp32 (for GELU').  Backward: dX = dY W^T (times GELU'(pre) of the layer
// below, fused), dW = X^T dY, db = column sums of dY.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "graf.h"

namespace graf {
unsigned int* device_error_word_address();  // graf_af.cu
}

namespace {

// GELU(x) = x Phi(x), Phi the standard normal CDF; GELU'(x) = Phi(x) + x phi(x).
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    const float pdf = 0.3989422804014327f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

__device__ __forceinline__ unsigned pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

enum Epi { EPI_BIAS_GELU = 0, EPI_BIAS = 1, EPI_DGELU = 2, EPI_STORE = 3 };

// C[M][N] = op(A) op(B) with
//   TA = false: A is [M][K] row-major (lda);  TA = true: A is stored [K][M] (lda)
//   TB = false: B is [K][N] row-major (ldb);  TB = true: B is stored [N][K] (ldb)
// Epilogues:
//   EPI_BIAS_GELU: pre = C + bias[n] -> out_f32 (pre), out_bf16 = bf16(GELU(pre))
//   EPI_BIAS:      out_f32 = C + bias[n]
//   EPI_DGELU:     out_bf16 = bf16(C * GELU'(aux[m][n]))   (aux: pre-activation below)
//   EPI_STORE:     out_f32 = C
//
// ------------------------------------------------------- tcgen05 / TMEM GEMM
// The GEMM runs on the 5th-generation tensor cores: one
// CTA of 4 warps per 128 x 64 tile of C; per 64-wide step of K, the threads
// stage A (128 rows of M) and B (64 rows of N), both K-major, in shared
// memory in the canonical layout without swizzle -- 8 x 8 core matrices of
// 128 B, core (row / 8, k / 8) at ((row / 8) (64 / 8) + k / 8) 128 B, with
// 16-byte loads and stores where k is the operand's contiguous index -- then
// one thread issues four tcgen05.mma.kind::f16 (M = 128, N = 64, K = 16,
// BF16 in, FP32 accumulated in tensor memory) and commits them to an
// mbarrier that every thread waits on before the tiles are refilled.  The
// accumulator (128 lanes x 64 columns of TMEM) is read back with tcgen05.ld,
// warp w owning lanes 32w .. 32w + 31 (rows of the tile), and goes through the
// epilogue.  Every wait is bounded (about a second of clock cycles); one that
// runs out sets GRAF_DEVERR_TIMEOUT in the device error word, and the CTA
// skips the rest, frees its tensor memory and returns.
constexpr int TC_BM = 128, TC_BN = 64, TC_BK = 64, TC_THREADS = 128;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;                  // 16 KB
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;                  // 8 KB
constexpr int TC_SMEM_LAUNCH = 29 * 1024;                      // at most 7 CTAs per SM: 7 x 64 <= 512 TMEM columns
constexpr long long TC_WAIT_CYCLES = 2000000000LL;             // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) of a K-major tile with 64 columns of K in
// the canonical no-swizzle layout.
__device__ __forceinline__ uint32_t core_offset(int row, int k) {
    return (uint32_t)((((row >> 3) * (TC_BK / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices adjacent in K), stride-dimension byte offset
// (between core matrices adjacent in M or N), the fixed version field
// (bits 46-48 = 1), no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bits
// 17-22, M / 16 at bits 24-28.
constexpr uint32_t umma_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Tile of ROWS x 64 from X with k contiguous (element (row, k) at
// X[(row0 + row) ld + k0 + k]): 8 consecutive k -- one row of a core matrix --
// per 16-byte load and store where the row is whole and aligned, elementwise
// at the edges.
template <int ROWS>
__device__ __forceinline__ void load_tile_k(const __nv_bfloat16* __restrict__ X, int ld, int row0, int nrows,
                                            int k0, int K, unsigned char* T, int tid) {
    const bool vec = (ld % 8 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    for (int e = tid; e < ROWS * (TC_BK / 8); e += TC_THREADS) {
        const int r = e / (TC_BK / 8), c = (e % (TC_BK / 8)) * 8;
        const int gr = row0 + r, gk = k0 + c;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gr < nrows) {
            if (vec && gk + 8 <= K) {
                v = *reinterpret_cast<const uint4*>(X + (size_t)gr * ld + gk);
            } else {
                unsigned w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int ka = gk + 2 * i, kb = ka + 1;
                    w[i] = pack_bf16(ka < K ? X[(size_t)gr * ld + ka] : __float2bfloat16(0.0f),
                                     kb < K ? X[(size_t)gr * ld + kb] : __float2bfloat16(0.0f));
                }
                v = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        *reinterpret_cast<uint4*>(T + core_offset(r, c)) = v;
    }
}

// Tile of ROWS x 64 from X with the row index contiguous (element (row, k) at
// X[(k0 + k) ld + row0 + row]): loads coalesce along the rows, stores are
// elementwise.
template <int ROWS>
__device__ __forceinline__ void load_tile_mn(const __nv_bfloat16* __restrict__ X, int ld, int row0, int nrows,
                                             int k0, int K, unsigned char* T, int tid) {
    for (int e = tid; e < ROWS * TC_BK; e += TC_THREADS) {
        const int r = e % ROWS, c = e / ROWS;
        const int gr = row0 + r, gk = k0 + c;
        const __nv_bfloat16 v = (gr < nrows && gk < K) ? X[(size_t)gk * ld + gr] : __float2bfloat16(0.0f);
        *reinterpret_cast<__nv_bfloat16*>(T + core_offset(r, c)) = v;
    }
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(TC_THREADS) gemm_tc_kernel(const __nv_bfloat16* __restrict__ A, int lda,
                                                              const __nv_bfloat16* __restrict__ B, int ldb, int M,
                                                              int N, int K, const float* __restrict__ bias,
                                                              const float* __restrict__ aux, int ldaux,
                                                              float* __restrict__ out_f32,
                                                              __nv_bfloat16* __restrict__ out_bf16, int ldo,
                                                              unsigned int* err) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* As = tc_smem;
    unsigned char* Bs = tc_smem + TC_A_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(tc_smem + TC_A_BYTES + TC_B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_smem + TC_A_BYTES + TC_B_BYTES + 8);
    volatile int* sflag = reinterpret_cast<volatile int*>(tc_smem + TC_A_BYTES + TC_B_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
    const uint32_t bar_a = smem_u32(bar);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *sflag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma_idesc(TC_BM, TC_BN);
    const int nk = (K + TC_BK - 1) / TC_BK;
    bool ok = true;
    for (int kc = 0; kc < nk && ok; ++kc) {
        const int k0 = kc * TC_BK;
        // A tile (row m, k); B tile, K-major: (row n, k) = op(B)[k][n]
        if (TA) load_tile_mn<TC_BM>(A, lda, m0, M, k0, K, As, tid);
        else load_tile_k<TC_BM>(A, lda, m0, M, k0, K, As, tid);
        if (TB) load_tile_k<TC_BN>(B, ldb, n0, N, k0, K, Bs, tid);
        else load_tile_mn<TC_BN>(B, ldb, n0, N, k0, K, Bs, tid);
        // the tiles, written by the generic proxy, become visible to the
        // tensor cores' (async proxy) reads
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
            for (int s = 0; s < TC_BK / 16; ++s)  // K = 16 per instruction: two core matrices along K
                umma_f16(tmem, umma_desc(a0 + s * 256, 128, (TC_BK / 8) * 128),
                         umma_desc(b0 + s * 256, 128, (TC_BK / 8) * 128), idesc, (kc > 0 || s > 0) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             bar_a)
                         : "memory");
            const long long t0 = clock64();
            while (!mbar_try_wait(bar_a, (uint32_t)(kc & 1))) {
                if (clock64() - t0 > TC_WAIT_CYCLES) {
                    *sflag = 1 + (kc & 1);  // the phase still awaited, plus one
                    atomicOr(err, GRAF_DEVERR_TIMEOUT);
                    break;
                }
            }
        }
        __syncthreads();
        ok = *sflag == 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        // this warp's 32 rows of the tile, 16 columns per load
        const int m = m0 + warp * 32 + lane;
        for (int j = 0; j < TC_BN / 16; ++j) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 16), v);
            if (m >= M) continue;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int n = n0 + j * 16 + c;
                if (n >= N) continue;
                const size_t o = (size_t)m * ldo + n;
                if constexpr (EPI == EPI_BIAS_GELU) {
                    const float pre = v[c] + bias[n];
                    out_f32[o] = pre;
                    out_bf16[o] = __float2bfloat16(gelu(pre));
                } else if constexpr (EPI == EPI_BIAS) {
                    out_f32[o] = v[c] + bias[n];
                } else if constexpr (EPI == EPI_DGELU) {
                    out_bf16[o] = __float2bfloat16(v[c] * gelu_grad(aux[(size_t)m * ldaux + n]));
                } else {
                    out_f32[o] = v[c];
                }
            }
        }
    }
    if (!ok && tid == 0) {
        // a wait ran out: give the MMAs in flight one more bounded wait
        // before their tensor memory is freed
        const long long t0 = clock64();
        while (!mbar_try_wait(bar_a, (uint32_t)(*sflag - 1)) && clock64() - t0 < TC_WAIT_CYCLES) {
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_BN) : "memory");
    }
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                 const float* bias, const float* aux, int ldaux, float* of, __nv_bfloat16* ob, int ldo,
                 cudaStream_t st) {
    unsigned int* err = graf::device_error_word_address();
    if (!err) return cudaErrorUnknown;
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<TA, TB, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TC_SMEM_LAUNCH);
    if (e != cudaSuccess) return e;
    dim3 grid((N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM);
    gemm_tc_kernel<TA, TB, EPI><<<grid, TC_THREADS, TC_SMEM_LAUNCH, st>>>(A, lda, B, ldb, M, N, K, bias, aux, ldaux,
                                                                          of, ob, ldo, err);
    return cudaGetLastError();
}

// Column sums (bias gradient) of a fp32 or bf16 [rows][cols] matrix, fixed order.
__global__ void colsum_kernel(const __nv_bfloat16* __restrict__ X, int rows, int cols, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += __bfloat162float(X[(size_t)r * cols + c]);
    out[c] = s;
}

__global__ void to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// Spec features [rows][8] fp32 -> bf16 [rows][16] (zero padded to the mma k-step).
__global__ void pack_input_kernel(const float* __restrict__ x, int rows, __nv_bfloat16* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * 16) return;
    const int r = i / 16, c = i % 16;
    y[i] = __float2bfloat16(c < GRAF_MLP_IN ? x[r * GRAF_MLP_IN + c] : 0.0f);
}

// Phase label loss per row b (invariant to a global phase and to conjugation,
// the symmetries that leave a masked ISL over |m| <= Mw unchanged):
//   z_s = (1/N) sum_n exp(j (p_n - s t_n)), s = +-1;  L_b = min_s (1 - |z_s|)
//   dL_b/dp_n = Im(conj(z) exp(j (p_n - s t_n))) / (N |z|) for the minimising s.
// One block per row; scale multiplies the gradient (e.g. 1 / rows for a mean),
// and the gradient is written in bf16 as the last layer's dY.
__global__ void phase_loss_kernel(const float* __restrict__ pred, const float* __restrict__ target, int rows,
                                  int n, float scale, float* __restrict__ loss, __nv_bfloat16* __restrict__ dpred) {
    const int b = blockIdx.x;
    const float* p = pred + (size_t)b * n;
    const float* t = target + (size_t)b * n;
    float zr[2] = {0.0f, 0.0f}, zi[2] = {0.0f, 0.0f};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float s0, c0, s1, c1;
        sincosf(p[i] - t[i], &s0, &c0);
        sincosf(p[i] + t[i], &s1, &c1);
        zr[0] += c0; zi[0] += s0;
        zr[1] += c1; zi[1] += s1;
    }
    __shared__ float red[4][32];
    for (int o = 16; o > 0; o >>= 1)
        for (int s = 0; s < 2; ++s) {
            zr[s] += __shfl_xor_sync(0xffffffffu, zr[s], o);
            zi[s] += __shfl_xor_sync(0xffffffffu, zi[s], o);
        }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = zr[0]; red[1][w] = zi[0]; red[2][w] = zr[1]; red[3][w] = zi[1];
    }
    __syncthreads();
    float a[4] = {0, 0, 0, 0};
    for (int k = 0; k < nw; ++k)
        for (int c = 0; c < 4; ++c) a[c] += red[c][k];
    const float inv_n = 1.0f / n;
    const float m0 = sqrtf(a[0] * a[0] + a[1] * a[1]) * inv_n, m1 = sqrtf(a[2] * a[2] + a[3] * a[3]) * inv_n;
    const int s = (m1 > m0) ? 1 : 0;  // sign -1 when conjugation matches better
    const float mag = s ? m1 : m0;
    const float zrr = (s ? a[2] : a[0]) * inv_n, zii = (s ? a[3] : a[1]) * inv_n;
    if (threadIdx.x == 0 && loss) loss[b] = 1.0f - mag;
    const float sg = s ? -1.0f : 1.0f;
    const float f = mag > 0.0f ? scale / (n * mag) : 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float sn, cs;
        sincosf(p[i] - sg * t[i], &sn, &cs);
        // Im(conj(z) e^{j theta}) = zr sin - zi cos
        dpred[(size_t)b * n + i] = __float2bfloat16(f * (zrr * sn - zii * cs));
    }
}

graf_status_t st_of(cudaError_t e) { return e == cudaSuccess ? GRAF_OK : GRAF_ERR_CUDA; }

}  // namespace

extern "C" {

size_t graf_mlp_param_count(void) {
    return (size_t)GRAF_MLP_IN_PAD * GRAF_MLP_HID + GRAF_MLP_HID + (size_t)GRAF_MLP_HID * GRAF_MLP_HID +
           GRAF_MLP_HID + (size_t)GRAF_MLP_HID * GRAF_MLP_OUT + GRAF_MLP_OUT;
}

size_t graf_mlp_activation_bytes(int32_t rows) {
    if (rows < 1) return 0;
    const size_t r = (size_t)rows;
    // x16 bf16, pre1/pre2 fp32, h1/h2 bf16, dy3 bf16, dpre2 / dpre1 bf16
    return r * GRAF_MLP_IN_PAD * 2 + 2 * r * GRAF_MLP_HID * 4 + 2 * r * GRAF_MLP_HID * 2 +
           r * GRAF_MLP_OUT * 2 + 2 * r * GRAF_MLP_HID * 2 + 1024;
}

graf_status_t graf_mlp_cast_params(const float* master, void* params_bf16, void* stream) {
    if (!master || !params_bf16) return GRAF_ERR_INVALID_ARG;
    const long long n = (long long)graf_mlp_param_count();
    to_bf16_kernel<<<256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        master, static_cast<__nv_bfloat16*>(params_bf16), n);
    return st_of(cudaGetLastError());
}

// Parameter layout (both fp32 master and bf16 copies): W1 [16][512] | b1 [512] |
// W2 [512][512] | b2 [512] | W3 [512][1024] | b3 [1024]; biases are read from
// the fp32 master copy.
struct Views {
    const __nv_bfloat16 *W1, *W2, *W3;
    const float *b1, *b2, *b3;
};
static Views views(const void* pb, const float* master) {
    const __nv_bfloat16* p = static_cast<const __nv_bfloat16*>(pb);
    Views v;
    size_t o = 0;
    v.W1 = p + o; o += (size_t)GRAF_MLP_IN_PAD * GRAF_MLP_HID;
    v.b1 = master + o; o += GRAF_MLP_HID;
    v.W2 = p + o; o += (size_t)GRAF_MLP_HID * GRAF_MLP_HID;
    v.b2 = master + o; o += GRAF_MLP_HID;
    v.W3 = p + o; o += (size_t)GRAF_MLP_HID * GRAF_MLP_OUT;
    v.b3 = master + o;
    return v;
}

struct Acts {
    __nv_bfloat16* x16;
    float *pre1, *pre2;
    __nv_bfloat16 *h1, *h2, *dy3, *dpre2, *dpre1;
};
static Acts acts(void* a, int rows) {
    unsigned char* p = static_cast<unsigned char*>(a);
    const size_t r = (size_t)rows;
    Acts s;
    s.x16 = reinterpret_cast<__nv_bfloat16*>(p); p += r * GRAF_MLP_IN_PAD * 2;
    s.pre1 = reinterpret_cast<float*>(p); p += r * GRAF_MLP_HID * 4;
    s.pre2 = reinterpret_cast<float*>(p); p += r * GRAF_MLP_HID * 4;
    s.h1 = reinterpret_cast<__nv_bfloat16*>(p); p += r * GRAF_MLP_HID * 2;
    s.h2 = reinterpret_cast<__nv_bfloat16*>(p); p += r * GRAF_MLP_HID * 2;
    s.dy3 = reinterpret_cast<__nv_bfloat16*>(p); p += r * GRAF_MLP_OUT * 2;
    s.dpre2 = reinterpret_cast<__nv_bfloat16*>(p); p += r * GRAF_MLP_HID * 2;
    s.dpre1 = reinterpret_cast<__nv_bfloat16*>(p);
    return s;
}

graf_status_t graf_mlp_forward(const float* spec, int32_t rows, const float* master, const void* params_bf16,
                               float* phases, void* activations, void* stream) {
    if (!spec || rows < 1 || !master || !params_bf16 || !phases || !activations) return GRAF_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Views v = views(params_bf16, master);
    const Acts a = acts(activations, rows);
    pack_input_kernel<<<(rows * 16 + 255) / 256, 256, 0, st>>>(spec, rows, a.x16);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = gemm<false, false, EPI_BIAS_GELU>(a.x16, GRAF_MLP_IN_PAD, v.W1, GRAF_MLP_HID, rows, GRAF_MLP_HID,
                                              GRAF_MLP_IN_PAD, v.b1, nullptr, 0, a.pre1, a.h1, GRAF_MLP_HID, st);
    if (e == cudaSuccess)
        e = gemm<false, false, EPI_BIAS_GELU>(a.h1, GRAF_MLP_HID, v.W2, GRAF_MLP_HID, rows, GRAF_MLP_HID,
                                              GRAF_MLP_HID, v.b2, nullptr, 0, a.pre2, a.h2, GRAF_MLP_HID, st);
    if (e == cudaSuccess)
        e = gemm<false, false, EPI_BIAS>(a.h2, GRAF_MLP_HID, v.W3, GRAF_MLP_OUT, rows, GRAF_MLP_OUT, GRAF_MLP_HID,
                                         v.b3, nullptr, 0, phases, nullptr, GRAF_MLP_OUT, st);
    return st_of(e);
}

graf_status_t graf_mlp_label_loss(const float* phases, const float* target, int32_t rows, float scale,
                                  float* loss, void* activations, void* stream) {
    if (!phases || !target || rows < 1 || !activations) return GRAF_ERR_INVALID_ARG;
    const Acts a = acts(activations, rows);
    phase_loss_kernel<<<rows, 256, 0, static_cast<cudaStream_t>(stream)>>>(phases, target, rows, GRAF_MLP_OUT,
                                                                           scale, loss, a.dy3);
    return st_of(cudaGetLastError());
}

graf_status_t graf_mlp_set_output_grad(const float* dphases, int32_t rows, void* activations, void* stream) {
    if (!dphases || rows < 1 || !activations) return GRAF_ERR_INVALID_ARG;
    const Acts a = acts(activations, rows);
    to_bf16_kernel<<<256, 256, 0, static_cast<cudaStream_t>(stream)>>>(dphases, a.dy3,
                                                                       (long long)rows * GRAF_MLP_OUT);
    return st_of(cudaGetLastError());
}

graf_status_t graf_mlp_backward(int32_t rows, const float* master, const void* params_bf16, void* activations,
                                float* grad, void* stream) {
    if (rows < 1 || !master || !params_bf16 || !activations || !grad) return GRAF_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Views v = views(params_bf16, master);
    const Acts a = acts(activations, rows);
    float* gW1 = grad;
    float* gb1 = gW1 + (size_t)GRAF_MLP_IN_PAD * GRAF_MLP_HID;
    float* gW2 = gb1 + GRAF_MLP_HID;
    float* gb2 = gW2 + (size_t)GRAF_MLP_HID * GRAF_MLP_HID;
    float* gW3 = gb2 + GRAF_MLP_HID;
    float* gb3 = gW3 + (size_t)GRAF_MLP_HID * GRAF_MLP_OUT;
    cudaError_t e;
    // layer 3: dW3 = h2^T dy3, db3 = sum dy3, dpre2 = (dy3 W3^T) * GELU'(pre2)
    e = gemm<true, false, EPI_STORE>(a.h2, GRAF_MLP_HID, a.dy3, GRAF_MLP_OUT, GRAF_MLP_HID, GRAF_MLP_OUT, rows,
                                     nullptr, nullptr, 0, gW3, nullptr, GRAF_MLP_OUT, st);
    if (e == cudaSuccess) {
        colsum_kernel<<<(GRAF_MLP_OUT + 255) / 256, 256, 0, st>>>(a.dy3, rows, GRAF_MLP_OUT, gb3);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = gemm<false, true, EPI_DGELU>(a.dy3, GRAF_MLP_OUT, v.W3, GRAF_MLP_OUT, rows, GRAF_MLP_HID, GRAF_MLP_OUT,
                                         nullptr, a.pre2, GRAF_MLP_HID, nullptr, a.dpre2, GRAF_MLP_HID, st);
    // layer 2
    if (e == cudaSuccess)
        e = gemm<true, false, EPI_STORE>(a.h1, GRAF_MLP_HID, a.dpre2, GRAF_MLP_HID, GRAF_MLP_HID, GRAF_MLP_HID, rows,
                                         nullptr, nullptr, 0, gW2, nullptr, GRAF_MLP_HID, st);
    if (e == cudaSuccess) {
        colsum_kernel<<<(GRAF_MLP_HID + 255) / 256, 256, 0, st>>>(a.dpre2, rows, GRAF_MLP_HID, gb2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = gemm<false, true, EPI_DGELU>(a.dpre2, GRAF_MLP_HID, v.W2, GRAF_MLP_HID, rows, GRAF_MLP_HID, GRAF_MLP_HID,
                                         nullptr, a.pre1, GRAF_MLP_HID, nullptr, a.dpre1, GRAF_MLP_HID, st);
    // layer 1 (input gradient not needed)
    if (e == cudaSuccess)
        e = gemm<true, false, EPI_STORE>(a.x16, GRAF_MLP_IN_PAD, a.dpre1, GRAF_MLP_HID, GRAF_MLP_IN_PAD,
                                         GRAF_MLP_HID, rows, nullptr, nullptr, 0, gW1, nullptr, GRAF_MLP_HID, st);
    if (e == cudaSuccess) {
        colsum_kernel<<<(GRAF_MLP_HID + 255) / 256, 256, 0, st>>>(a.dpre1, rows, GRAF_MLP_HID, gb1);
        e = cudaGetLastError();
    }
    return st_of(e);
}

}  // extern "C"
