// graf_kernels.cuh - launch parameters and shared device helpers of the
// ambiguity-function kernels.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "graf_fft.cuh"

namespace graf {

constexpr int kThreads = 256;     // threads per CTA of the row kernels (RowPlan<M>::THREADS for the largest M)

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount),
// read at every call; 152 (a GB300) only when no CUDA device is visible, so that
// workspace sizes can still be queried on a host without a GPU.
int device_sm_count();

// Per-waveform parameters of a batch of unequal waveforms (device table, one
// entry per waveform).  Offsets are in elements of the arrays they index.
struct WaveDesc {
    long long x_off;      // first element of waveform b in the packed input
    long long out_off;    // first element of its gradient in the packed output
    long long af_off;     // first float of its window in the packed forward output
    long long gpart_off;  // first float2 of its per-CTA gradient partials (tiles x N)
    int rec_off;          // index of its first per-CTA record / scale / sum
    int N, M;
    int k_lo, k_hi, m_lo, m_hi, k_ml, m_ml;
    int r_lo, r_hi, rows_per_tile, tiles, defer_hi;
    int unscaled;         // 1: its gradient partials are final (loss, then recomputing backward)
    float eps, beta, w_psl, w_isl;
};

// Everything a row kernel needs, passed by value.  Two modes: a uniform
// batch (waves == nullptr: B waveforms of length N sharing window and loss,
// CTA i handles waveform i / tiles, tile i % tiles) or a batch plan (waves
// and items set: persistent CTAs claim work items (waveform, tile) from an
// atomic counter in the order the plan gives, longest first).
struct AfParams {
    const void* x;   // uniform: [B][N]; plan: packed, waveform b at waves[b].x_off
    int kind;        // 0 complex, 1 phase
    int B, N, M;     // plan: N = longest waveform, M = this launch's row length
    int k_lo, k_hi, m_lo, m_hi, k_ml, m_ml;
    int r_lo, r_hi;        // k >= 0 rows to transform (negative rows are mirrored)
    int rows_per_tile, tiles;
    int full_m;            // window covers every Doppler bin
    float eps, beta, w_psl, w_isl;
    float* af_out;         // forward: [B][k_hi-k_lo+1][m_hi-m_lo+1]
    float4* rec;           // loss: per-CTA records {isl, max, sum, T}
    float* out8;           // loss: [B][8] scalars
    const float* saved8;   // backward: [B][8]
    float2* gpart;         // backward: per-CTA partial dL/ds*
    float* csum;           // backward: per-CTA sum of c a2
    double* usum;          // backward (grad_s): per waveform {sum_k w_b(k) (C[k] + eps), E} [B][2]
    int phase_only;        // backward: only dL/dphi is wanted (row k = 0 contributes nothing)
    int acc_copies;        // backward: gradient accumulators per CTA (divides the slot count)
    // fused loss + gradient
    int defer_hi;          // rows r_lo..defer_hi get loss partials only (their gradient is
                           // computed by af_backward_kernel after the loss is known); -1: none
    float* scale;          // per-CTA gradient scale, written by the loss finalisation
    // gradient reduction: a second set of partials (deferred rows), unscaled (uniform mode)
    int tiles2;
    const float2* gpart2;  // [B][tiles2][N]
    const float* csum2;    // [B][tiles2]
    // periodic AF (the paper's own definition, Eq. 7): circular lag mod N,
    // M = N; the signal and the gradient accumulators are stored twice in
    // shared memory so that s[(n-k) mod N] = s2[n - k + N] needs no index
    // wrap.  pconj: the +j exponent of Eq. 7, computed as the -j transform of
    // conj(s) (|X| and the losses are the same; the gradients are mapped back).
    int periodic, pconj;
    int chi_out;           // forward output: 0 Ahat, 1 |X|^2 / E^2, 2 |X|^2
    // match to a target surface (L_match of Eq. 22)
    const float* target;   // [B][k_hi-k_lo+1][m_hi-m_lo+1] target Ahat^2 over the window
    float match_w;         // its weight lambda_1
    float* mpart;          // per-CTA partial sums of (Ahat^2 - target)^2
    int grad_acc;          // gradient reduction adds to the output instead of writing it
    // batch plan
    const WaveDesc* waves;
    const int2* items;     // (waveform, tile) of this launch's work items, longest first
    int n_items;
    unsigned int* counter; // zeroed before the launch
    // hard PSL (beta = +inf): per waveform {transformed row k >= 0 of the
    // arg-max cell (-1: Omega empty), its DFT bin q in [0, M), float bits of
    // max Ahat^2, 0}, written by the loss finalisation (nullable)
    int4* peak;
};

// Spectral variance of the normalised power spectrum (the LPI term of the
// experiment loss, Sec. 7.1.1 Eq. 25), one row slot per waveform.
struct SpecParams {
    const void* x;   // [B][N] phases (kind 1) or complex64 (kind 0)
    int kind, B, N;
    float weight;    // its weight in the loss (lambda alpha)
    float* out8;     // nullable: out8[b][0] += weight SV, out8[b][7] = SV
    float* sv;       // nullable: SV [B]
    float2* grad_s;  // nullable: += or = weight * 2 dSV/ds*
    float* grad_phi; // nullable: += or = weight * dSV/dphi
    int accumulate;
};
cudaError_t run_spectral(const SpecParams& q, cudaStream_t st);

// Two terms of the composite loss (Sec. 5.1, Eq. 22) from the zero-Doppler
// autocorrelation and the modulus: W = sum_k |k| sigmoid(gamma (a2[k] - 1/2))
// and V = var(|s|), one row slot per waveform on a row of M = nextpow2(2N).
struct CompParams {
    const void* x;
    int kind, B, N;
    float gamma, eps, w_width, w_const;
    float* out8;     // nullable: out8[b][0] += w_width W + w_const V
    float* terms;    // nullable: [B][2] = {W, V}
    float2* grad_s;  // nullable: += or = 2 dL/ds*
    float* grad_phi; // nullable: += or = dL/dphi
    int accumulate;
};
cudaError_t run_composite(const CompParams& q, int M, cudaStream_t st);
template <int M> cudaError_t run_match_m(const AfParams& p, cudaStream_t st);
cudaError_t run_match(const AfParams& p, float* loss_out, cudaStream_t st);
template <int M> cudaError_t run_composite_m(const CompParams& q, cudaStream_t st);
template <int M> cudaError_t run_spectral_m(const SpecParams& q, cudaStream_t st);

// Shared-memory length of the signal: N, or 2N for the periodic AF (the
// signal twice, so that s[(n - k) mod N] is one load).
__host__ __device__ __forceinline__ int sig_len(const AfParams& p) { return p.periodic ? 2 * p.N : p.N; }
// Host and device mirror of RowPlan<M>::TPR: threads per row.
__host__ __device__ __forceinline__ int tpr_of(int M) {
    return M >= 512 ? M / 32 : (M >= 128 ? M / 16 : (M < 64 ? 1 : M / 64));
}

// Elements (float or float2) from one gradient accumulator of a CTA to the
// next: N, plus TPR when a warp holds several row slots (TPR < 32), so that
// the slots of one warp, which use consecutive accumulators, fall in
// different shared-memory banks.
__host__ __device__ __forceinline__ int acc_stride(int N, int tpr) { return N + (tpr < 32 ? tpr : 0); }

// Bytes of all gradient accumulators of a CTA (256-byte aligned).
__host__ __device__ __forceinline__ size_t acc_region_bytes(const AfParams& p) {
    return ((size_t)p.acc_copies * acc_stride(p.N, tpr_of(p.M)) * (p.phase_only ? sizeof(float) : sizeof(float2)) +
            255) &
           ~(size_t)255;
}

// The view of one waveform a kernel works with, in either mode.
struct Wave {
    const void* x;  // this waveform's input
    long long out_off, gpart_off;
    long long af_off;  // first float of its window in the forward output
    int rec_off;
    int kind, N, M;
    int k_lo, k_hi, m_lo, m_hi, k_ml, m_ml;
    int r_lo, r_hi, rows_per_tile, tiles, full_m, defer_hi, unscaled;
    int periodic, pconj;
    int sN;         // shared-memory length of the signal: N, or 2N periodic
    float eps, beta, w_psl, w_isl;
    // Hard PSL (the loss's beta = +inf): L = w_peak max_Omega Ahat^2 + w_isl ISL.
    // The view then carries beta = 0 and w_psl = 0, so that the kernels' soft
    // log-sum-exp term vanishes and they compute ISL and the maximum; the
    // maximum's gradient is added through its arg-max cell (peak_grad_kernel).
    int hard;
    float w_peak;
    // Fixed log-sum-exp shift (in units of Ahat^2), 0 = none.  For phase
    // input E = N and every cell has a2 = |X|^2/E^2 + eps/E^2 <= 1 + eps/N^2
    // (|X[k,m]| <= E by Cauchy-Schwarz), so with m = (1 + eps/N^2)/2 the terms
    // exp(beta (a2 - m)) stay within 2^(+-88) whenever beta log2(e) m <= 88:
    // no running maximum is needed.  Per-CTA loss records hold their sums
    // relative to this shift when it is set, else relative to their maximum.
    float lse_fix;
};

// beta = +inf selects the hard PSL (larger than any finite float).
__host__ __device__ __forceinline__ bool is_hard_beta(float beta) { return beta > 3.4028234e38f; }

// The fixed log-sum-exp shift of a waveform (see Wave::lse_fix), 0 = none.
// Host code uses it too: with a fixed shift no accumulator is ever rescaled,
// so the fused PSL path may share gradient accumulators between row slots.
__host__ __device__ __forceinline__ float lse_fixed_shift(int kind, float eps, float beta, int N) {
    if (kind != 1) return 0.0f;
    const float m = 0.5f * (1.0f + eps / ((float)N * (float)N));
    return beta * 1.4426950408889634f * m <= 88.0f ? m : 0.0f;
}

__host__ __device__ __forceinline__ Wave wave_of(const AfParams& p, int b) {
    Wave w;
    w.kind = p.kind;
    if (p.waves) {
        const WaveDesc& d = p.waves[b];
        w.x = static_cast<const char*>(p.x) + d.x_off * (p.kind == 1 ? 4 : 8);
        w.out_off = d.out_off;
        w.gpart_off = d.gpart_off;
        w.af_off = d.af_off;
        w.rec_off = d.rec_off;
        w.N = d.N; w.M = d.M;
        w.k_lo = d.k_lo; w.k_hi = d.k_hi; w.m_lo = d.m_lo; w.m_hi = d.m_hi; w.k_ml = d.k_ml; w.m_ml = d.m_ml;
        w.r_lo = d.r_lo; w.r_hi = d.r_hi; w.rows_per_tile = d.rows_per_tile; w.tiles = d.tiles;
        w.defer_hi = d.defer_hi;
        w.unscaled = d.unscaled;
        w.eps = d.eps; w.beta = d.beta; w.w_psl = d.w_psl; w.w_isl = d.w_isl;
        w.periodic = 0;
        w.pconj = 0;
    } else {
        w.x = static_cast<const char*>(p.x) + (long long)b * p.N * (p.kind == 1 ? 4 : 8);
        w.out_off = (long long)b * p.N;
        w.gpart_off = (long long)b * p.tiles * p.N;
        w.af_off = (long long)b * (p.k_hi - p.k_lo + 1) * (p.m_hi - p.m_lo + 1);
        w.rec_off = b * p.tiles;
        w.N = p.N; w.M = p.M;
        w.k_lo = p.k_lo; w.k_hi = p.k_hi; w.m_lo = p.m_lo; w.m_hi = p.m_hi; w.k_ml = p.k_ml; w.m_ml = p.m_ml;
        w.r_lo = p.r_lo; w.r_hi = p.r_hi; w.rows_per_tile = p.rows_per_tile; w.tiles = p.tiles;
        w.defer_hi = p.defer_hi;
        w.unscaled = 0;
        w.eps = p.eps; w.beta = p.beta; w.w_psl = p.w_psl; w.w_isl = p.w_isl;
        w.periodic = p.periodic;
        w.pconj = p.pconj;
    }
    w.sN = w.periodic ? 2 * w.N : w.N;
    w.full_m = (w.m_lo == -(w.M / 2) && w.m_hi == w.M / 2 - 1) ? 1 : 0;
    w.hard = is_hard_beta(w.beta) ? 1 : 0;
    w.w_peak = w.hard ? w.w_psl : 0.0f;
    if (w.hard) {
        w.beta = 0.0f;
        w.w_psl = 0.0f;
    }
    w.lse_fix = lse_fixed_shift(w.kind, w.eps, w.beta, w.N);
    return w;
}

// Base weight w_b(k) of transformed row k >= 0 (see the backward kernel): the
// weight every Doppler bin of rows k and -k carries when the window spans all
// bins, unless the mainlobe box takes half the row or more; otherwise 0.
__host__ __device__ __forceinline__ int base_weight(const Wave& w, int k) {
    if (!w.full_m) return 0;
    if (k <= w.k_ml && 2 * w.m_ml + 1 > w.M / 2) return 0;
    return ((k >= w.k_lo && k <= w.k_hi) ? 1 : 0) + ((k > 0 && -k >= w.k_lo && -k <= w.k_hi) ? 1 : 0);
}

// Row range and tiling shared by the host code (workspace sizes) and launches.
struct Tiling {
    int r_lo, r_hi, nrows, slots, rows_per_tile, tiles;
};

// Host mirrors of RowPlan<M>: threads per CTA and row slots (tpr_of above).
inline int threads_of(int M) { return tpr_of(M) > 256 ? tpr_of(M) : 256; }
inline int slots_of(int M) { return threads_of(M) / tpr_of(M); }

constexpr size_t kMaxSmem = 232448;  // opt-in dynamic shared memory per CTA (227 KB)
constexpr size_t kSmemPerSm = 233472;  // shared memory per SM (228 KB)
constexpr size_t kRedBytes = 1024;   // block-reduction scratch

template <int M>
__host__ __device__ constexpr size_t smem_signal_bytes(int N) {
    return ((size_t)N * sizeof(float2) + 255) & ~(size_t)255;
}
template <int M, int V = 0>
__host__ __device__ constexpr size_t row_buffer_bytes() {
    using P = RowPlan<M, V>;
    return (((size_t)P::SMEM_ROW * (P::SPLIT ? sizeof(float) : sizeof(float2)) * (P::THREADS / P::TPR)) + 255) &
           ~(size_t)255;
}
template <int M>
constexpr size_t forward_smem(int N) {
    return smem_signal_bytes<M>(N) + row_buffer_bytes<M>() + kRedBytes;
}
// Gradient accumulators: complex (float2) in general, real (float) when only
// the phase gradient is wanted (see scatter_row_real).
// per: periodic AF (the signal is stored twice; accumulators keep N entries).
template <int M, int V = 0>
constexpr size_t backward_smem(int N, int acc_copies, int real = 0, int per = 0) {
    return smem_signal_bytes<M>(per ? 2 * N : N) + row_buffer_bytes<M, V>() +
           (((size_t)acc_copies * acc_stride(N, RowPlan<M>::TPR) * (real ? sizeof(float) : sizeof(float2)) + 255) &
            ~(size_t)255) +
           kRedBytes;
}
// Number of gradient accumulators per CTA (a power of two <= slots; slots
// sharing one take turns in the scatter): the largest that still lets the
// registers' number of CTAs share an SM, if that leaves at most two turns,
// else the largest that fits in shared memory; 0 if even one does not.
template <int M>
int backward_acc_copies(int N, int real = 0, int per = 0) {
    constexpr int slots = RowPlan<M>::THREADS / RowPlan<M>::TPR;
    constexpr int per_sm = RowPlan<M>::MIN_BLOCKS;
    if (per_sm > 1) {
        const size_t budget = kSmemPerSm / per_sm - 1024;  // 1 KB per CTA is reserved
        for (int a = slots; a >= 1 && 2 * a >= slots; a /= 2)
            if (backward_smem<M>(N, a, real, per) <= budget) return a;
    }
    for (int a = slots; a >= 1; a /= 2)
        if (backward_smem<M>(N, a, real, per) <= kMaxSmem) return a;
    return 0;
}

size_t row_kernel_smem(int M, int N, int which);  // which: 0 forward/loss, 2 backward
cudaError_t run_loss_rows(const AfParams& p, cudaStream_t st);      // loss row kernel only
cudaError_t run_backward_rows(const AfParams& p, cudaStream_t st);  // backward row kernel only
int acc_copies_for(int M, int N, int real = 0, int per = 0);  // backward accumulators, 0 = unsupported
template <int M> cudaError_t run_forward_m(const AfParams& p, cudaStream_t st);
template <int M> cudaError_t run_loss_m(const AfParams& p, cudaStream_t st);
template <int M> cudaError_t run_backward_m(const AfParams& p, cudaStream_t st);
template <int M> cudaError_t run_fused_m(const AfParams& p, cudaStream_t st);
cudaError_t run_fused(const AfParams& p, cudaStream_t st);
cudaError_t run_finalize(const AfParams& p, cudaStream_t st);
// Hard PSL: add (accumulate != 0) or write dL w_peak dAhat^2[peak]/d(s or phi)
// for every waveform from the peak records of the finalisation.
cudaError_t run_peak_grad(const AfParams& p, const float* dL, float2* grad_s, float* grad_phi, int accumulate,
                          cudaStream_t st);
cudaError_t run_grad_reduce(const AfParams& p, const float* dL, float2* grad_s, float* grad_phi,
                            cudaStream_t st);
cudaError_t run_forward(const AfParams& p, cudaStream_t st);
cudaError_t run_loss(const AfParams& p, cudaStream_t st);
cudaError_t run_backward(const AfParams& p, const float* dL, float2* grad_s, float* grad_phi,
                         cudaStream_t st);

// Tiles of transformed rows [r_lo, r_hi] for B waveforms: rows per CTA a
// multiple of the slot count, at least 4 CTAs per SM (of `sms` SMs) where the
// batch allows.
inline Tiling make_tiling_rows(int B, int M, int r_lo, int r_hi, int sms) {
    Tiling T;
    T.r_lo = r_lo;
    T.r_hi = r_hi;
    T.nrows = T.r_hi - T.r_lo + 1;
    T.slots = slots_of(M);
    // up to 512 rows per tile over 64 slots' worth of threads (16 rows per slot
    // when a row has 32 values per thread, 8 when it has 64)
    int rps = M >= 128 ? 16 : 8;
    while (rps > 1) {
        long long tiles = (T.nrows + (long long)T.slots * rps - 1) / ((long long)T.slots * rps);
        if ((long long)B * tiles >= 4LL * sms) break;
        rps /= 2;
    }
    T.rows_per_tile = T.slots * rps;
    T.tiles = (T.nrows + T.rows_per_tile - 1) / T.rows_per_tile;
    return T;
}

// Rows k >= 0 whose transform serves the window: row k gives delay k and,
// by |X[-k,m]| = |X[k,-m]|, delay -k.
inline Tiling make_tiling(int B, int M, int k_lo, int k_hi, int sms) {
    if (k_lo >= 0) return make_tiling_rows(B, M, k_lo, k_hi, sms);
    if (k_hi <= 0) return make_tiling_rows(B, M, -k_hi, -k_lo, sms);
    return make_tiling_rows(B, M, 0, (-k_lo > k_hi) ? -k_lo : k_hi, sms);
}

// ex2.approx (PTX): 2^x with relative error below 2^-22, +0 at -inf.
__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The same, kept in program order: inside a long unrolled loop the scheduler
// would otherwise issue every exponential early and hold all the results.
__device__ __forceinline__ float ex2v(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Load s[0..N) of one waveform into shared memory (phases -> exp(j phi)) and
// return E = sum |s|^2, reduced in a fixed order (identical in every CTA).
__device__ __forceinline__ float load_signal(const Wave& wv, float2* s_sm, float* red) {
    const int tid = threadIdx.x;
    float e = 0.0f;
    if (wv.kind == 1) {
        const float* ph = static_cast<const float*>(wv.x);
        for (int n = tid; n < wv.N; n += (int)blockDim.x) {
            float sn, cs;
            sincosf(__ldg(ph + n), &sn, &cs);
            const float2 v = make_float2(cs, wv.pconj ? -sn : sn);
            s_sm[n] = v;
            if (wv.periodic) s_sm[n + wv.N] = v;
            e = fmaf(cs, cs, fmaf(sn, sn, e));
        }
    } else {
        const float2* xs = static_cast<const float2*>(wv.x);
        for (int n = tid; n < wv.N; n += (int)blockDim.x) {
            float2 v = __ldg(xs + n);
            if (wv.pconj) v.y = -v.y;
            s_sm[n] = v;
            if (wv.periodic) s_sm[n + wv.N] = v;
            e = fmaf(v.x, v.x, fmaf(v.y, v.y, e));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((tid & 31) == 0) red[tid >> 5] = e;
    __syncthreads();
    float E = 0.0f;
#pragma unroll
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) E += red[w];
    __syncthreads();
    return E;
}

// Doppler index (fftshift order) of register w of thread t.
template <int M>
__device__ __forceinline__ int doppler_of(int t, int w) {
    using P = RowPlan<M>;
    const int q = t + P::TPR * w;
    return (w >= P::VALS / 2) ? q - M : q;
}

// Loss weights.  A transformed cell (k >= 0, Doppler m) stands for (k, m)
// and, for k > 0, the mirrored (-k, -m); its weight is the number of those in
// Omega (0, 1 or 2).  The Doppler tests depend only on the thread, so they
// are packed once per CTA into 64-bit column masks (bit w = register w):
struct ColMasks {
    unsigned long long in_m;   // m in [m_lo, m_hi]
    unsigned long long in_mm;  // mirrored Doppler in [m_lo, m_hi]
    unsigned long long ml_m;   // |m| <= m_ml
};

template <int M>
__device__ __forceinline__ ColMasks col_masks(const Wave& p, int t) {
    using P = RowPlan<M>;
    ColMasks c{0ull, 0ull, 0ull};
    for (int w = 0; w < P::VALS; ++w) {
        const int q = t + P::TPR * w;
        const int m = (w >= P::VALS / 2) ? q - M : q;
        const int mm = (m == -(M / 2)) ? m : -m;
        const int am = m < 0 ? -m : m;
        const unsigned long long bit = 1ull << w;
        if (m >= p.m_lo && m <= p.m_hi) c.in_m |= bit;
        if (mm >= p.m_lo && mm <= p.m_hi) c.in_mm |= bit;
        if (am <= p.m_ml) c.ml_m |= bit;
    }
    return c;
}

// Per-row masks: bit w of `one` = weight >= 1, of `two` = weight 2.  Also the
// plain window masks of rows k and -k for the forward store.
struct RowMasks {
    unsigned long long pos, neg, one, two;
};

__device__ __forceinline__ RowMasks row_masks(const Wave& p, const ColMasks& c, int k) {
    const bool in_pos = (k >= p.k_lo) && (k <= p.k_hi);
    const bool in_neg = (k > 0) && (-k >= p.k_lo) && (-k <= p.k_hi);
    const bool ml_row = k <= p.k_ml;  // k >= 0, so |-k| = k too
    RowMasks r;
    r.pos = in_pos ? c.in_m : 0ull;
    r.neg = in_neg ? c.in_mm : 0ull;
    const unsigned long long keep = ml_row ? ~c.ml_m : ~0ull;
    r.one = (r.pos | r.neg) & keep;
    r.two = (r.pos & r.neg) & keep;
    return r;
}

template <int W>
__device__ __forceinline__ bool mbit(unsigned long long m) {
    if constexpr (W < 32) return (static_cast<unsigned>(m) >> W) & 1u;
    else return (static_cast<unsigned>(m >> 32) >> (W - 32)) & 1u;
}

template <int W>
__device__ __forceinline__ float mweight(const RowMasks& r) {
    return (mbit<W>(r.one) ? 1.0f : 0.0f) + (mbit<W>(r.two) ? 1.0f : 0.0f);
}

}  // namespace graf
