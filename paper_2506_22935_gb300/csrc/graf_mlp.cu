// graf_mlp.cu - the learned proposal network: an MLP that maps a design spec
// to initial phase codes (the "neural network -> waveform -> GRAF layer ->
// loss" pipeline of the paper's Sec. 6.1), trained and run entirely by these
// kernels.  BF16 operands on the tensor cores (mma.sync m16n8k16), FP32
// accumulation, FP32 master weights.
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

namespace {

constexpr int BM = 64, BN = 64, BK = 16;  // CTA tile
constexpr int PAD = 8;                    // bf16 elements of row padding in shared memory

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

// D = A B + D for one 16x8x16 tile (PTX mma.sync, row.col, bf16 -> f32).
__device__ __forceinline__ void mma16816(float* d, const unsigned* a, const unsigned* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
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
// 4 warps, each a 32x32 sub-tile (2 x 4 mma tiles); K stepped by 16 through
// shared memory, where A is kept [m][k] and B [n][k] (k contiguous), the
// fragment orders of mma.sync's row.col form.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __nv_bfloat16* __restrict__ A, int lda,
                                                         const __nv_bfloat16* __restrict__ B, int ldb, int M,
                                                         int N, int K, const float* __restrict__ bias,
                                                         const float* __restrict__ aux, int ldaux,
                                                         float* __restrict__ out_f32,
                                                         __nv_bfloat16* __restrict__ out_bf16, int ldo) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, q = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    for (int k0 = 0; k0 < K; k0 += BK) {
        // 64 x 16 elements of each operand, 8 per thread
        for (int e = tid; e < BM * BK; e += 128) {
            const int r = e / BK, c = e % BK;
            const int gm = m0 + r, gk = k0 + c;
            As[r][c] = (gm < M && gk < K) ? (TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : zero;
            const int gn = n0 + r;
            Bs[r][c] = (gn < N && gk < K) ? (TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]) : zero;
        }
        __syncthreads();
        unsigned af[2][4], bf[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + i * 16 + g;
            af[i][0] = pack_bf16(As[r][2 * q], As[r][2 * q + 1]);
            af[i][1] = pack_bf16(As[r + 8][2 * q], As[r + 8][2 * q + 1]);
            af[i][2] = pack_bf16(As[r][2 * q + 8], As[r][2 * q + 9]);
            af[i][3] = pack_bf16(As[r + 8][2 * q + 8], As[r + 8][2 * q + 9]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = wn + j * 8 + g;
            bf[j][0] = pack_bf16(Bs[c][2 * q], Bs[c][2 * q + 1]);
            bf[j][1] = pack_bf16(Bs[c][2 * q + 8], Bs[c][2 * q + 9]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bf[j]);
        __syncthreads();
    }
    // epilogue: acc[i][j] holds rows g, g+8 and columns 2q, 2q+1 of tile (i, j)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * q + (r & 1);
                if (m >= M || n >= N) continue;
                const float c = acc[i][j][r];
                const size_t o = (size_t)m * ldo + n;
                if constexpr (EPI == EPI_BIAS_GELU) {
                    const float pre = c + bias[n];
                    out_f32[o] = pre;
                    out_bf16[o] = __float2bfloat16(gelu(pre));
                } else if constexpr (EPI == EPI_BIAS) {
                    out_f32[o] = c + bias[n];
                } else if constexpr (EPI == EPI_DGELU) {
                    out_bf16[o] = __float2bfloat16(c * gelu_grad(aux[(size_t)m * ldaux + n]));
                } else {
                    out_f32[o] = c;
                }
            }
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                 const float* bias, const float* aux, int ldaux, float* of, __nv_bfloat16* ob, int ldo,
                 cudaStream_t st) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    gemm_bf16_kernel<TA, TB, EPI><<<grid, 128, 0, st>>>(A, lda, B, ldb, M, N, K, bias, aux, ldaux, of, ob, ldo);
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
