// graf_af_impl.cuh - the ambiguity-function row kernels (forward store, fused
// losses, backward with recomputation) as templates over the row length M;
// graf_af_m*.cu instantiate them, a few M per translation unit.
//
// One CTA = RowPlan<M>::THREADS threads (256; 512 for M = 16384) = THREADS/TPR
// row slots; a CTA owns one waveform b and a
// tile of consecutive delay rows k >= 0.  Per row a slot builds the aperiodic
// lag product (Eq. 8) from the waveform in shared memory, transforms it
// (Eq. 11) with row_fft, and consumes the result in registers.  Rows k < 0
// are never transformed: |X[-k, m]| = |X[k, -m]|, so row k also serves delay
// -k with the Doppler axis mirrored (the loss weight of a transformed cell
// counts both cells, and its adjoint adds both).
#pragma once
#include <climits>

#include <math_constants.h>

#include "graf_kernels.cuh"

namespace graf {


// --------------------------------------------------------------- lag product
// v[w] = R[k, n] = s[n] conj(s[n - k]) for n = t + TPR w, support k <= n < N
// (k >= 0), zero elsewhere (Eq. 8, aperiodic).  HALF: N <= M/2, so registers
// w >= VALS/2 are zero and never touched.
template <int M, bool HALF>
__device__ __forceinline__ void build_lag_row(float2* v, const float2* s_sm, int N, int k, int t,
                                              bool valid) {
    using P = RowPlan<M>;
    constexpr int WN = HALF ? P::VALS / 2 : P::VALS;
    sfor<0, WN>([&](auto w) {
        const int n = t + P::TPR * decltype(w)::value;
        float2 r = make_float2(0.0f, 0.0f);
        // k <= n < N as one unsigned compare that depends on k (not hoistable)
        if (valid && (unsigned)(n - k) < (unsigned)(N - k)) r = cmulc(s_sm[n], s_sm[n - k]);
        v[w] = r;
    });
    if constexpr (HALF) {
        sfor<WN, P::VALS>([&](auto w) { v[w] = make_float2(0.0f, 0.0f); });
    }
}

// Work-item loop of a row kernel.  Uniform batch: CTA i runs item
// (i / tiles, i % tiles) once.  Batch plan: persistent CTAs claim items from
// the plan's atomic counter until none is left (items are ordered longest
// first, so this is a longest-processing-time schedule).
template <class F>
__device__ __forceinline__ void for_each_item(const AfParams& p, F&& body) {
    if (!p.items) {
        body((int)(blockIdx.x / p.tiles), (int)(blockIdx.x % p.tiles));
        return;
    }
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(p.counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= p.n_items) break;
        const int2 bt = p.items[it];
        body(bt.x, bt.y);
        __syncthreads();
    }
}

template <int M, bool HALF>
__device__ __forceinline__ void forward_item(const AfParams& p, int b, int tile, unsigned char* smem) {
    using P = RowPlan<M>;
    __shared__ Wave s_wave;
    if (threadIdx.x == 0) s_wave = wave_of(p, b);
    __syncthreads();
    const Wave& wv = s_wave;
    float2* s_sm = reinterpret_cast<float2*>(smem);
    float2* bufs = reinterpret_cast<float2*>(smem + smem_signal_bytes<M>(sig_len(p)));
    float* red = reinterpret_cast<float*>(smem + smem_signal_bytes<M>(sig_len(p)) + row_buffer_bytes<M>());

    const int tid = threadIdx.x, slot = tid / P::TPR, t = tid % P::TPR;
    const float E = load_signal(wv, s_sm, red);
    const float invE = 1.0f / E;
    const float sc = p.chi_out == 1 ? invE * invE : 1.0f;  // chi output: |X|^2 / E^2 or |X|^2
    float2* buf = bufs + (size_t)slot * (P::SPLIT ? P::SMEM_ROW / 2 : P::SMEM_ROW);
    const ColMasks cm = col_masks<M>(wv, t);

    const int ncols = wv.m_hi - wv.m_lo + 1;
    float* out_b = p.af_out + wv.af_off;
    const int row0 = wv.r_lo + tile * wv.rows_per_tile;
    const int row_end = min(row0 + wv.rows_per_tile, wv.r_hi + 1);
    // iterations for the rows this tile actually holds (CTA-uniform)
    const int iters = max(0, row_end - row0 + (P::THREADS / P::TPR) - 1) / (P::THREADS / P::TPR);

    float2 v[P::VALS];
    for (int it = 0; it < iters; ++it) {
        const int k = row0 + slot + it * (P::THREADS / P::TPR);
        const bool valid = k < row_end;
        build_lag_row<M, HALF>(v, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, valid);
        row_sync<P::TPR>(slot);
        row_fft<M, false, HALF, false>(v, buf, t, slot);
        if (valid) {
            const RowMasks rmk = row_masks(wv, cm, k);
            const bool in_pos = rmk.pos != 0ull, in_neg = rmk.neg != 0ull;
            // row k at rp[m], row -k at rn[m'] (m' = -m, and -M/2 maps to itself)
            float* rp = out_b + (in_pos ? (size_t)(k - wv.k_lo) * ncols : 0) - wv.m_lo + t;
            float* rn = out_b + (in_neg ? (size_t)(-k - wv.k_lo) * ncols : 0) - wv.m_lo - t;
            sfor<0, P::VALS>([&](auto w) {
                constexpr int W = decltype(w)::value;
                constexpr int off = P::TPR * W - (W >= P::VALS / 2 ? M : 0);  // m - t
                const float2 x = v[w];
                // sqrt(q) as q rsqrt(q) (one special-function op; relative
                // error ~2e-7, against the 1e-5 bound on Ahat <= 1)
                const float q = fmaf(x.x, x.x, fmaf(x.y, x.y, wv.eps));
                const float a = p.chi_out == 0 ? (q > 0.0f ? q * rsqrtf(q) * invE : 0.0f)
                                               : fmaf(x.x, x.x, x.y * x.y) * sc;
                if (mbit<W>(rmk.pos)) __stcs(rp + off, a);
                if (mbit<W>(rmk.neg)) {
                    float* dst = rn - off;
                    if constexpr (W == P::VALS / 2) {
                        if (t == 0) dst = rn + t - M / 2;
                    }
                    __stcs(dst, a);
                }
            });
        }
    }
}

// ---------------------------------------------------------- forward (store)
// Ahat = sqrt(|X|^2 + eps) / E (Eq. 12, Eq. 17) -- or chi = |X|^2 (Eq. 12,
// Algorithm 1), optionally over chi[0,0] = E^2 = max chi (Eq. 17) --
// for every window cell of rows k and -k.  Stores are coalesced along m
// (consecutive threads hold consecutive Doppler bins) and streaming (written
// once, never re-read here).  Uniform batches and batch plans alike (the
// window of waveform b starts at its af_off).
template <int M, bool HALF>
__global__ void __launch_bounds__(RowPlan<M>::THREADS, RowPlan<M>::MIN_BLOCKS) af_forward_kernel(AfParams p) {
    extern __shared__ __align__(256) unsigned char smem[];
    for_each_item(p, [&](int b, int tile) { forward_item<M, HALF>(p, b, tile, smem); });
}

// ---------------------------------------------------------- fused loss
// Per cell a2 = Ahat^2 = (|X|^2 + eps) / E^2 and weight w in {0,1,2}:
//   ISL += w a2;  hard max of a2 over weighted cells;
//   log-sum-exp of beta a2 kept as (running max mx, sum of exp(beta (a2 - mx)))
//   plus T = sum w exp(beta (a2 - mx)) a2 for the energy gradient.
// Per CTA one record {ISL, mx, sum, T} -> workspace.
__device__ __forceinline__ void lse_rescale(float& mx, float& sum, float& T, float new_mx, float bl2) {
    if (new_mx > mx) {
        const float f = ex2a((mx - new_mx) * bl2);
        sum *= f;
        T *= f;
        mx = new_mx;
    }
}

__device__ __forceinline__ void lse_merge(float& isl, float& mx, float& sum, float& T, float isl2,
                                          float mx2, float sum2, float T2, float bl2) {
    isl += isl2;
    if (mx2 > mx) {
        const float f = ex2a((mx - mx2) * bl2);
        sum = sum * f + sum2;
        T = T * f + T2;
        mx = mx2;
    } else if (mx2 > -CUDART_INF_F) {
        const float f = ex2a((mx2 - mx) * bl2);
        sum += sum2 * f;
        T += T2 * f;
    }
}

// Hard PSL: a candidate arg-max cell (value, transformed row, cell code) and
// the order that picks one: the larger value, then the smaller row, then the
// smaller code.  Every reduction below applies it, so the choice depends on
// the values alone.
struct PeakKey {
    float v;
    int row, code;
};

__device__ __forceinline__ bool peak_better(const PeakKey& a, const PeakKey& b) {
    return a.v > b.v || (a.v == b.v && (a.row < b.row || (a.row == b.row && a.code < b.code)));
}

__device__ __forceinline__ PeakKey warp_best(PeakKey k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const PeakKey c{__shfl_xor_sync(0xffffffffu, k.v, o), __shfl_xor_sync(0xffffffffu, k.row, o),
                        __shfl_xor_sync(0xffffffffu, k.code, o)};
        if (peak_better(c, k)) k = c;
    }
    return k;
}

// The CTA's best key, returned to every thread; `scratch` holds 3 words per
// warp.  Starts and ends with a barrier.
__device__ __forceinline__ PeakKey block_best(PeakKey k, float* scratch) {
    __syncthreads();
    k = warp_best(k);
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    if (lane == 0) {
        scratch[3 * wi] = k.v;
        scratch[3 * wi + 1] = __int_as_float(k.row);
        scratch[3 * wi + 2] = __int_as_float(k.code);
    }
    __syncthreads();
    PeakKey best{scratch[0], __float_as_int(scratch[1]), __float_as_int(scratch[2])};
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        const PeakKey c{scratch[3 * w], __float_as_int(scratch[3 * w + 1]), __float_as_int(scratch[3 * w + 2])};
        if (peak_better(c, best)) best = c;
    }
    __syncthreads();
    return best;
}

template <int M, bool HALF>
__device__ __forceinline__ void loss_item(const AfParams& p, int b, int tile, unsigned char* smem) {
    using P = RowPlan<M>;
    // the waveform's parameters live in shared memory (CTA-uniform), so they
    // are re-read after barriers instead of occupying registers
    __shared__ Wave s_wave;
    if (threadIdx.x == 0) s_wave = wave_of(p, b);
    __syncthreads();
    const Wave& wv = s_wave;
    float2* s_sm = reinterpret_cast<float2*>(smem);
    float2* bufs = reinterpret_cast<float2*>(smem + smem_signal_bytes<M>(sig_len(p)));
    float* red = reinterpret_cast<float*>(smem + smem_signal_bytes<M>(sig_len(p)) + row_buffer_bytes<M>());

    const int tid = threadIdx.x, slot = tid / P::TPR, t = tid % P::TPR;
    const float E = load_signal(wv, s_sm, red);
    if (tile == 0 && tid == 0) p.out8[(size_t)b * 8 + 4] = E;
    const float invE2 = 1.0f / (E * E);
    const float eps_n = wv.eps * invE2;
    const float bl2 = wv.beta * 1.4426950408889634f;  // beta * log2(e)
    float2* buf = bufs + (size_t)slot * (P::SPLIT ? P::SMEM_ROW / 2 : P::SMEM_ROW);
    const ColMasks cm = col_masks<M>(wv, t);
    constexpr unsigned long long full_mask = P::VALS == 64 ? ~0ull : ((1ull << P::VALS) - 1ull);

    const int row0 = wv.r_lo + tile * wv.rows_per_tile;
    const int row_end = min(row0 + wv.rows_per_tile, wv.r_hi + 1);
    constexpr int SLOTS = P::THREADS / P::TPR;
    // iterations for the rows this tile actually holds (CTA-uniform)
    const int iters = max(0, row_end - row0 + SLOTS - 1) / SLOTS;

    float isl = 0.0f, mx = -CUDART_INF_F, sum = 0.0f, T = 0.0f;
    // hard PSL: this thread's largest weighted a2, its row and bin (the first
    // bin of the first row that reached it)
    float hbest = -CUDART_INF_F;
    int hrow = INT_MAX, hq = INT_MAX;
    float2 v[P::VALS];
    for (int it = 0; it < iters; ++it) {
        const int k = row0 + slot + it * SLOTS;
        const bool valid = k < row_end;
        build_lag_row<M, HALF>(v, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, valid);
        row_sync<P::TPR>(slot);
        row_fft<M, false, HALF, false>(v, buf, t, slot);
        if (!valid) continue;
        const RowMasks rmk = row_masks(wv, cm, k);
        if ((rmk.one | rmk.two) == 0ull) continue;
        // a row whose weights are all equal (every Doppler bin in the window,
        // no mainlobe cell) skips the per-cell mask tests
        const bool uniform = rmk.one == full_mask && (rmk.two == 0ull || rmk.two == full_mask);
        const float wrow = rmk.two != 0ull ? 2.0f : 1.0f;
        // pass 1: a2, ISL, masked max (a2 overwrites v[w].x; v[w].y = weight)
        float rmx = -CUDART_INF_F, risl = 0.0f;
        sfor<0, P::VALS>([&](auto w) {
            const float2 x = v[w];
            const float a2 = fmaf(fmaf(x.x, x.x, x.y * x.y), invE2, eps_n);
            const float wt = uniform ? wrow : mweight<decltype(w)::value>(rmk);
            risl = fmaf(wt, a2, risl);
            rmx = fmaxf(rmx, wt > 0.0f ? a2 : -CUDART_INF_F);
            v[w] = make_float2(a2, wt);
        });
        if (rmx == -CUDART_INF_F) continue;
        isl += risl;
        if (wv.hard) {  // the maximum only; no log-sum-exp
            if (rmx > hbest) {
                hbest = rmx;
                hrow = k;
                hq = INT_MAX;
                sfor<0, P::VALS>([&](auto w) {
                    if (hq == INT_MAX && v[w].y > 0.0f && v[w].x == rmx) hq = t + P::TPR * decltype(w)::value;
                });
            }
            continue;
        }
        lse_rescale(mx, sum, T, rmx, bl2);
        const float sh = mx * bl2;
        sfor<0, P::VALS>([&](auto w) {
            const float a2 = v[w].x, wt = v[w].y;
            const float e = wt * ex2a(fmaf(a2, bl2, -sh));
            sum += e;
            T = fmaf(e, a2, T);
        });
    }
    // CTA reduction in a fixed order: warp xor tree, then warps 0..7
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float i2 = __shfl_xor_sync(0xffffffffu, isl, o);
        const float m2 = __shfl_xor_sync(0xffffffffu, mx, o);
        const float s2 = __shfl_xor_sync(0xffffffffu, sum, o);
        const float t2 = __shfl_xor_sync(0xffffffffu, T, o);
        lse_merge(isl, mx, sum, T, i2, m2, s2, t2, bl2);
    }
    float4* wred = reinterpret_cast<float4*>(red);
    if ((tid & 31) == 0) wred[tid >> 5] = make_float4(isl, mx, sum, T);
    __syncthreads();
    if (tid == 0) {
        float4 a = wred[0];
        for (int w = 1; w < P::THREADS / 32; ++w) {
            const float4 c = wred[w];
            lse_merge(a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w, bl2);
        }
        if (wv.lse_fix > 0.0f && a.y > -CUDART_INF_F) {  // sums relative to the fixed shift
            const float f = ex2a((a.y - wv.lse_fix) * bl2);
            a.z *= f;
            a.w *= f;
        }
        if (!wv.hard) p.rec[wv.rec_off + tile] = a;
        else red[120] = a.x;
    }
    if (wv.hard) {  // record {ISL, max, row, bin} of the CTA's arg-max cell
        const PeakKey pk = block_best(PeakKey{hbest, hrow, hq}, red + 64);
        if (tid == 0)
            p.rec[wv.rec_off + tile] = make_float4(red[120], pk.v, __int_as_float(pk.row), __int_as_float(pk.code));
    }
}

template <int M, bool HALF>
__global__ void __launch_bounds__(RowPlan<M>::THREADS, RowPlan<M>::MIN_BLOCKS) af_loss_kernel(AfParams p) {
    extern __shared__ __align__(256) unsigned char smem[];
    for_each_item(p, [&](int b, int tile) { loss_item<M, HALF>(p, b, tile, smem); });
}

// ---------------------------------------------------------- backward
// Per row: recompute X, form the cell adjoint, take the adjoint DFT
// (conjugate twiddles, unnormalised) and scatter both Wirtinger terms of
// R[k,n] = s[n] conj(s[n-k]) into this slot's accumulator:
//   acc[n]   += G_R[n] s[n-k]          (through conj(R), which carries s*[n])
//   acc[n-k] += conj(G_R[n]) s[n]       (through R, which carries s*[n-k])
// The two scatters run in separate phases so no two threads of a row update
// one address at once.  Slots then sum in a fixed order into one partial.
//
// Cell adjoint.  dL/dAhat^2 = w (w_isl + w_psl p), p = exp(beta (a2 -
// PSL_soft)), w the cell weight.  With p0 = exp(-beta PSL_soft), A' = w_isl +
// w_psl p0 and the row's base weight w_b (the weight every Doppler bin of the
// row has when the window spans all of them, else 0):
//   dL/dAhat^2 = w_b A'  +  [(w - w_b) A' + w w_psl (p - p0)].
// The first term is uniform over the row; its adjoint DFT is exactly
// w_b A' M R[k,n] / E^2 (the adjoint of an M-point DFT applied to the DFT of
// a row of support <= M is M times the row), whose scatter is s[p] times a
// real number: it contributes exactly nothing to dL/dphi, and for dL/ds it
// is added in closed form, in FP64, by grad_s_kernel.  Only the second
// term goes through the FFT, G = c X with c = [...] / E^2.  This keeps the
// PSL term, whose softmax weights are ~1/|Omega| (2.4e-7 at N=1024, M=2048),
// from vanishing next to the ISL weight in FP32, and avoids summing the
// ISL gradient of full rows (zero for unit modulus, by Parseval) from large
// cancelling parts.  Per CTA the kernel also sums c a2 for the energy term.
// Scatter both Wirtinger terms of R[k,n] = s[n] conj(s[n-k]) for row k from
// G_R (in v, natural strided layout) into the slot's accumulator:
//   acc[n]   += G_R[n] s[n-k]     (through conj(R), which carries s*[n])
//   acc[n-k] += conj(G_R[n]) s[n]  (through R, which carries s*[n-k])
// in two phases so no two threads of a row update one address at once.
// Slots that share an accumulator (turns > 1) take turns, CTA-wide.
// CONJ: v holds Y = conj(G_R) (the adjoint computed as conj(DFT(conj(G)))):
// G_R s = cmulc(s, Y) and conj(G_R) s = Y s.
// wrap (periodic AF, lag k - N, N = M a power of two): the second index n - k
// lies in [N - k, 2N - k) and is taken mod N, so one N-length accumulator
// serves both terms.
template <int M, bool HALF, bool CONJ = false>
__device__ __forceinline__ void scatter_row(const float2* v, float2* acc, const float2* s_sm, int N,
                                            int k, int t, bool active, int slot, int turns,
                                            int my_turn, bool wrap) {
    using P = RowPlan<M>;
    constexpr int WN = HALF ? P::VALS / 2 : P::VALS;
    auto scatter_a = [&]() {
        if (!active) return;
        sfor<0, WN>([&](auto w) {
            const int n = t + P::TPR * decltype(w)::value;
            if ((unsigned)(n - k) < (unsigned)(N - k)) {
                const float2 a = acc[n];
                const float2 g = CONJ ? cmulc(s_sm[n - k], v[w]) : cmul(v[w], s_sm[n - k]);
                acc[n] = cadd(a, g);
            }
        });
    };
    // (N = M, a power of two, for the periodic AF; HALF rows have 2N <= M,
    // which no periodic row has)
    const int wrap_mask = (!HALF && wrap) ? N - 1 : -1;
    auto scatter_b = [&]() {
        if (!active) return;
        sfor<0, WN>([&](auto w) {
            const int n = t + P::TPR * decltype(w)::value;
            if ((unsigned)(n - k) < (unsigned)(N - k)) {
                const int i = HALF ? n - k : (n - k) & wrap_mask;
                const float2 a = acc[i];
                const float2 g = CONJ ? cmul(v[w], s_sm[n]) : cmulc(s_sm[n], v[w]);
                acc[i] = cadd(a, g);
            }
        });
    };
    if (turns == 1) {
        scatter_a();
        row_sync<P::TPR>(slot);
        scatter_b();
        row_sync<P::TPR>(slot);
    } else {
        for (int tt = 0; tt < turns; ++tt) {
            if (tt == my_turn) scatter_a();
            __syncthreads();
        }
        for (int tt = 0; tt < turns; ++tt) {
            if (tt == my_turn) scatter_b();
            __syncthreads();
        }
    }
}

// Phase-only gradient with a real accumulator.  grad_phi[p] = 2 Im(g[p]
// s*[p]) and the two Wirtinger terms of row k give
//   Im(G_R[k,n] s[n-k] s*[n]) = q[k,n]          at p = n,
//   Im(conj(G_R[k,n]) s[n] s*[n-k]) = -q[k,n]   at p = n - k,
// with q = Im(G_R conj(R)), R[k,n] = s[n] conj(s[n-k]) (Eq. 8): one real
// number per cell, added at n and subtracted at n - k.  v holds conj(G_R)
// (CONJ form), so q = -Im(v R).  Row 0 cancels exactly (n = n - k).
template <int M, bool HALF>
__device__ __forceinline__ void scatter_row_real(const float2* v, float* acc, const float2* s_sm, int N,
                                                 int k, int t, bool active, int slot, int turns,
                                                 int my_turn, bool wrap) {
    using P = RowPlan<M>;
    constexpr int WN = HALF ? P::VALS / 2 : P::VALS;
    float q[WN];
    sfor<0, WN>([&](auto w) {
        const int n = t + P::TPR * decltype(w)::value;
        q[w] = 0.0f;
        if (active && (unsigned)(n - k) < (unsigned)(N - k)) {
            const float2 r = cmulc(s_sm[n], s_sm[n - k]);
            q[w] = -fmaf(v[w].x, r.y, v[w].y * r.x);
        }
    });
    auto scatter_a = [&]() {
        if (!active) return;
        sfor<0, WN>([&](auto w) {
            const int n = t + P::TPR * decltype(w)::value;
            if ((unsigned)(n - k) < (unsigned)(N - k)) acc[n] += q[w];
        });
    };
    const int wrap_mask = (!HALF && wrap) ? N - 1 : -1;  // periodic: index mod N (N = M)
    auto scatter_b = [&]() {
        if (!active) return;
        sfor<0, WN>([&](auto w) {
            const int n = t + P::TPR * decltype(w)::value;
            if ((unsigned)(n - k) < (unsigned)(N - k)) {
                const int i = HALF ? n - k : (n - k) & wrap_mask;
                acc[i] -= q[w];
            }
        });
    };
    if (turns == 1) {
        scatter_a();
        row_sync<P::TPR>(slot);
        scatter_b();
        row_sync<P::TPR>(slot);
    } else {
        for (int tt = 0; tt < turns; ++tt) {
            if (tt == my_turn) scatter_a();
            __syncthreads();
        }
        for (int tt = 0; tt < turns; ++tt) {
            if (tt == my_turn) scatter_b();
            __syncthreads();
        }
    }
}

// Per-CTA partial sums of the gradient accumulators and one scalar, in a
// fixed order (warp xor tree, then warps in order).  Phase-only mode: the
// accumulators are real (copy i at floats [i N, (i+1) N)) and a partial is
// stored as (sum, 0).
template <int M, int V = 0>
__device__ __forceinline__ void write_grad_partial(const AfParams& p, const Wave& wv, const float2* acc_all,
                                                   float* red, float cs, int tile) {
    using P = RowPlan<M, V>;
    const int tid = threadIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
    if ((tid & 31) == 0) red[tid >> 5] = cs;
    __syncthreads();
    if (tid == 0) {
        float s = red[0];
        for (int w = 1; w < P::THREADS / 32; ++w) s += red[w];
        p.csum[wv.rec_off + tile] = s;
    }
    float2* out = p.gpart + wv.gpart_off + (long long)tile * wv.N;
    if (p.phase_only) {
        const float* acc_r = reinterpret_cast<const float*>(acc_all);
        for (int n = tid; n < wv.N; n += P::THREADS) {
            float a = acc_r[n];
            for (int s = 1; s < p.acc_copies; ++s) a += acc_r[(size_t)s * acc_stride(wv.N, P::TPR) + n];
            out[n] = make_float2(a, 0.0f);
        }
        return;
    }
    for (int n = tid; n < wv.N; n += P::THREADS) {
        float2 a = acc_all[n];
        for (int s = 1; s < p.acc_copies; ++s) a = cadd(a, acc_all[(size_t)s * acc_stride(wv.N, P::TPR) + n]);
        out[n] = a;
    }
}

template <int M, bool HALF, bool RO>
__device__ __forceinline__ void backward_item(const AfParams& p, int b, int tile, unsigned char* smem) {
    const bool phase_only = RO || p.phase_only;  // RO: only dL/dphi is wanted, known at compile time
    using P = RowPlan<M>;
    constexpr int SLOTS = P::THREADS / P::TPR;
    // the waveform's parameters live in shared memory (CTA-uniform), so they
    // are re-read after barriers instead of occupying registers
    __shared__ Wave s_wave;
    if (threadIdx.x == 0) s_wave = wave_of(p, b);
    __syncthreads();
    const Wave& wv = s_wave;
    float2* s_sm = reinterpret_cast<float2*>(smem);
    float2* bufs = reinterpret_cast<float2*>(smem + smem_signal_bytes<M>(sig_len(p)));
    float2* acc_all = reinterpret_cast<float2*>(smem + smem_signal_bytes<M>(sig_len(p)) + row_buffer_bytes<M>());
    float* red = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(acc_all) +
                                          acc_region_bytes(p));

    const int tid = threadIdx.x, slot = tid / P::TPR, t = tid % P::TPR;
    for (int i = tid; i < (int)(acc_region_bytes(p) / sizeof(float2)); i += P::THREADS)
        acc_all[i] = make_float2(0.0f, 0.0f);
    const float E = load_signal(wv, s_sm, red);  // includes __syncthreads
    // the item's constants live in shared memory and are re-read after the
    // forward transform, so that none of them occupies a register during it
    __shared__ float s_c[7];
    if (tid == 0) {
        const float invE2 = 1.0f / (E * E);
        const float bl2 = wv.beta * 1.4426950408889634f;
        const float psl_soft = p.saved8[(size_t)b * 8 + 1];
        const float sh = psl_soft * bl2;
        const float p0 = ex2a(-sh);
        s_c[0] = invE2;
        s_c[1] = wv.eps * invE2;                         // eps / E^2
        s_c[2] = bl2;
        s_c[3] = sh;
        s_c[4] = p0;
        s_c[5] = fmaf(wv.w_psl, p0, wv.w_isl) * invE2;  // cA = A' / E^2
        s_c[6] = wv.w_psl * invE2;                       // cP
    }
    __syncthreads();
    float csum = 0.0f;
    float2* buf = bufs + (size_t)slot * (P::SPLIT ? P::SMEM_ROW / 2 : P::SMEM_ROW);
    const ColMasks cm = col_masks<M>(wv, t);
    constexpr unsigned long long full_mask = P::VALS == 64 ? ~0ull : ((1ull << P::VALS) - 1ull);
    // slots sharing an accumulator (when shared memory is short) take turns
    const int turns = SLOTS / p.acc_copies;
    const int my_turn = slot / p.acc_copies;
    float2* acc = acc_all + (size_t)(slot % p.acc_copies) * acc_stride(wv.N, P::TPR);
    float* acc_r = reinterpret_cast<float*>(acc_all) + (size_t)(slot % p.acc_copies) * acc_stride(wv.N, P::TPR);

    const int row0 = wv.r_lo + tile * wv.rows_per_tile;
    const int row_end = min(row0 + wv.rows_per_tile, wv.r_hi + 1);
    // iterations for the rows this tile actually holds (CTA-uniform)
    const int iters = max(0, row_end - row0 + SLOTS - 1) / SLOTS;

    float2 v[P::VALS];
    for (int it = 0; it < iters; ++it) {
        const int k = row0 + slot + it * SLOTS;
        // row 0 is R[0,n] = |s[n]|^2: it does not depend on the phases
        const bool valid = k < row_end && !(phase_only && k == 0);
        build_lag_row<M, HALF>(v, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, valid);
        // one transform instance, run twice: recompute X, then the adjoint as
        // conj(DFT(conj(c X)))
#pragma unroll 1
        for (int ph = 0; ph < 2; ++ph) {
            row_sync<P::TPR>(slot);
            row_fft<M, false, false, false>(v, buf, t, slot);
            if (ph == 1) break;
            const float invE2 = s_c[0], eps_n = s_c[1], bl2 = s_c[2], sh = s_c[3], p0 = s_c[4], cA = s_c[5],
                        cP = s_c[6];
            const RowMasks rmk = row_masks(wv, cm, k);
            const bool uniform = rmk.one == full_mask && (rmk.two == 0ull || rmk.two == full_mask);
            const float wrow = valid ? (rmk.two != 0ull ? 2.0f : (rmk.one != 0ull ? 1.0f : 0.0f)) : 0.0f;
            const float wb = valid ? (float)base_weight(wv, k) : 0.0f;
            // registers with weight 0 and no row-uniform part (wb = 0) have
            // c = 0: skipped (the same registers on every lane for a Doppler band)
            const unsigned long long need = !valid ? 0ull : (wb != 0.0f ? full_mask : rmk.one);
            sfor<0, P::VALS>([&](auto w) {
                if (!mbit<decltype(w)::value>(need)) {
                    v[w] = make_float2(0.0f, 0.0f);
                    return;
                }
                const float2 x = v[w];
                const float a2 = fmaf(fmaf(x.x, x.x, x.y * x.y), invE2, eps_n);
                const float wt = (uniform || !valid) ? wrow : mweight<decltype(w)::value>(rmk);
                const float pr = ex2a(fmaf(a2, bl2, -sh));
                const float cpsl = wt > 0.0f ? wt * cP * (pr - p0) : 0.0f;
                float c = fmaf(wt - wb, cA, cpsl);
                // the origin X[0,0] = E: its scatter (2 E c s) and energy term
                // (-2 E c a2 s) cancel to -2 eps c s / E, added in closed form by
                // grad_s_kernel; leaving it out here avoids the cancellation
                if constexpr (decltype(w)::value == 0) {
                    if (k == 0 && t == 0) c = 0.0f;
                }
                csum = fmaf(c, a2, csum);
                v[w] = make_float2(c * x.x, -c * x.y);
            });
        }
        if (phase_only) {
            scatter_row_real<M, HALF>(v, acc_r, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, valid, slot, turns,
                                      my_turn, wv.periodic != 0);
        } else if constexpr (!RO) {
            scatter_row<M, HALF, true>(v, acc, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, valid, slot, turns,
                                       my_turn, wv.periodic != 0);
        }
    }
    write_grad_partial<M>(p, wv, acc_all, red, csum, tile);
}

template <int M, bool HALF, bool RO>
__global__ void __launch_bounds__(RowPlan<M>::THREADS, RowPlan<M>::MIN_BLOCKS) af_backward_kernel(AfParams p) {
    extern __shared__ __align__(256) unsigned char smem[];
    for_each_item(p, [&](int b, int tile) { backward_item<M, HALF, RO>(p, b, tile, smem); });
}

// ---------------------------------------------------------- match to a target
// L = lambda_1 sum_window (Ahat^2[k,m] - target[k,m])^2 (L_match of Eq. 22,
// on the energy-normalised chi / chi(0,0) of Eq. 17).  Its cell adjoint is
// local: c = 2 lambda_1 (Ahat^2 - target) / E^2 summed over the cell and its
// mirror, so one pass per row recomputes X, forms c X, takes the adjoint DFT
// and scatters (as the backward kernel), and adds the row's loss partial.
template <int M, bool HALF>
__device__ __forceinline__ void match_item(const AfParams& p, int b, int tile, unsigned char* smem) {
    using P = RowPlan<M>;
    constexpr int SLOTS = P::THREADS / P::TPR;
    __shared__ Wave s_wave;
    if (threadIdx.x == 0) s_wave = wave_of(p, b);
    __syncthreads();
    const Wave& wv = s_wave;
    float2* s_sm = reinterpret_cast<float2*>(smem);
    float2* bufs = reinterpret_cast<float2*>(smem + smem_signal_bytes<M>(sig_len(p)));
    float2* acc_all = reinterpret_cast<float2*>(smem + smem_signal_bytes<M>(sig_len(p)) + row_buffer_bytes<M>());
    float* red = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(acc_all) +
                                          acc_region_bytes(p));
    const int tid = threadIdx.x, slot = tid / P::TPR, t = tid % P::TPR;
    for (int i = tid; i < (int)(acc_region_bytes(p) / sizeof(float2)); i += P::THREADS)
        acc_all[i] = make_float2(0.0f, 0.0f);
    const float E = load_signal(wv, s_sm, red);  // includes __syncthreads
    const float invE2 = 1.0f / (E * E);
    const float eps_n = wv.eps * invE2;
    const float c2 = 2.0f * p.match_w * invE2;
    float2* buf = bufs + (size_t)slot * (P::SPLIT ? P::SMEM_ROW / 2 : P::SMEM_ROW);
    const ColMasks cm = col_masks<M>(wv, t);
    const int turns = SLOTS / p.acc_copies;
    const int my_turn = slot / p.acc_copies;
    float2* acc = acc_all + (size_t)(slot % p.acc_copies) * acc_stride(wv.N, P::TPR);
    float* acc_r = reinterpret_cast<float*>(acc_all) + (size_t)(slot % p.acc_copies) * acc_stride(wv.N, P::TPR);
    const int ncols = wv.m_hi - wv.m_lo + 1;
    const float* tgt = p.target + (size_t)b * (wv.k_hi - wv.k_lo + 1) * ncols;

    const int row0 = wv.r_lo + tile * wv.rows_per_tile;
    const int row_end = min(row0 + wv.rows_per_tile, wv.r_hi + 1);
    const int iters = max(0, row_end - row0 + SLOTS - 1) / SLOTS;
    float msum = 0.0f, csum = 0.0f;
    float2 v[P::VALS];
    for (int it = 0; it < iters; ++it) {
        const int k = row0 + slot + it * SLOTS;
        const bool valid = k < row_end;
        // row 0 is R[0,n] = |s[n]|^2: its loss counts, its phase gradient is 0
        const bool grad_row = valid && !(p.phase_only && k == 0);
        build_lag_row<M, HALF>(v, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, valid);
#pragma unroll 1
        for (int ph = 0; ph < 2; ++ph) {
            row_sync<P::TPR>(slot);
            row_fft<M, false, false, false>(v, buf, t, slot);
            if (ph == 1) break;
            const RowMasks rmk = row_masks(wv, cm, k);
            // row k at tp[m], row -k at tn[-m] (m = -M/2 maps to itself)
            const float* tp = tgt + (rmk.pos ? (size_t)(k - wv.k_lo) * ncols : 0) - wv.m_lo;
            const float* tn = tgt + (rmk.neg ? (size_t)(-k - wv.k_lo) * ncols : 0) - wv.m_lo;
            sfor<0, P::VALS>([&](auto w) {
                constexpr int W = decltype(w)::value;
                const int m = doppler_of<M>(t, W);
                const float2 x = v[w];
                const float a2 = fmaf(fmaf(x.x, x.x, x.y * x.y), invE2, eps_n);
                float d = 0.0f;
                if (valid && mbit<W>(rmk.pos)) {
                    const float dp = a2 - __ldg(tp + m);
                    msum = fmaf(dp, dp, msum);
                    d += dp;
                }
                if (valid && mbit<W>(rmk.neg)) {
                    const float dn = a2 - __ldg(tn + (m == -(M / 2) ? m : -m));
                    msum = fmaf(dn, dn, msum);
                    d += dn;
                }
                const float c = grad_row ? c2 * d : 0.0f;
                csum = fmaf(c, a2, csum);
                v[w] = make_float2(c * x.x, -c * x.y);
            });
            if constexpr (P::TPR >= 32) {
                if (!grad_row) break;  // slot-uniform
            }
        }
        if (p.phase_only)
            scatter_row_real<M, HALF>(v, acc_r, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, grad_row, slot, turns,
                                      my_turn, wv.periodic != 0);
        else
            scatter_row<M, HALF, true>(v, acc, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, grad_row, slot, turns,
                                       my_turn, wv.periodic != 0);
    }
    // the tile's loss partial, fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, o);
    if ((tid & 31) == 0) red[64 + (tid >> 5)] = msum;
    __syncthreads();
    if (tid == 0) {
        float s = red[64];
        for (int w = 1; w < P::THREADS / 32; ++w) s += red[64 + w];
        p.mpart[wv.rec_off + tile] = s;
    }
    write_grad_partial<M>(p, wv, acc_all, red, csum, tile);
}

template <int M, bool HALF>
__global__ void __launch_bounds__(RowPlan<M>::THREADS, RowPlan<M>::MIN_BLOCKS) af_match_kernel(AfParams p) {
    extern __shared__ __align__(256) unsigned char smem[];
    for_each_item(p, [&](int b, int tile) { match_item<M, HALF>(p, b, tile, smem); });
}

// ---------------------------------------------------------- fused loss + gradient
// Maximum over the TPR threads of one row slot (slots are contiguous thread
// ranges: a segment of a warp, one warp, or several warps).
template <int TPR>
__device__ __forceinline__ float slot_max(float x, float* scratch, int slot) {
    if constexpr (TPR <= 32) {
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
        return x;
    } else {
        constexpr int WPS = TPR / 32;  // warps per slot
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
        const int wi = (threadIdx.x % TPR) >> 5;
        float* sc = scratch + slot * WPS;
        if ((threadIdx.x & 31) == 0) sc[wi] = x;
        row_sync<TPR>(slot);
        float m = sc[0];
#pragma unroll
        for (int i = 1; i < WPS; ++i) m = fmaxf(m, sc[i]);
        row_sync<TPR>(slot);
        return m;
    }
}

// Sum over the TPR threads of one row slot, in a fixed order.
template <int TPR>
__device__ __forceinline__ float slot_sum(float x, float* scratch, int slot) {
    if constexpr (TPR <= 32) {
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        return x;
    } else {
        constexpr int WPS = TPR / 32;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        const int wi = (threadIdx.x % TPR) >> 5;
        float* sc = scratch + slot * WPS;
        if ((threadIdx.x & 31) == 0) sc[wi] = x;
        row_sync<TPR>(slot);
        float s = sc[0];
#pragma unroll
        for (int i = 1; i < WPS; ++i) s += sc[i];
        row_sync<TPR>(slot);
        return s;
    }
}

// ---------------------------------------------------------- spectral variance
// One row slot per waveform (N = M):
//   S = DFT_N(s), P = |S|^2, q = P / sum P, SV = (1/N) sum (q - 1/N)^2
//   dSV/dP[g] = (2 / (N sum P)) (q[g] - sum_f q[f]^2)
//             = (2 / (N sum P)) ((q[g] - 1/N) - N SV)        (no cancellation)
//   dSV/ds*[n] = sum_g dSV/dP[g] S[g] exp(+j 2 pi g n / N)  (adjoint DFT, run
//                as conj(DFT(conj(.))) on the same transform instance)
template <int M>
__global__ void __launch_bounds__(RowPlan<M>::THREADS, RowPlan<M>::MIN_BLOCKS) spectral_kernel(SpecParams q) {
    using P = RowPlan<M>;
    constexpr int SLOTS = P::THREADS / P::TPR;
    extern __shared__ __align__(256) unsigned char smem[];
    float2* bufs = reinterpret_cast<float2*>(smem);
    float* red = reinterpret_cast<float*>(smem + row_buffer_bytes<M>());
    const int tid = threadIdx.x, slot = tid / P::TPR, t = tid % P::TPR;
    const int b = blockIdx.x * SLOTS + slot;
    const bool valid = b < q.B;  // slot-uniform
    float2* buf = bufs + (size_t)slot * (P::SPLIT ? P::SMEM_ROW / 2 : P::SMEM_ROW);
    float2 v[P::VALS];
    sfor<0, P::VALS>([&](auto w) {
        const int n = t + P::TPR * decltype(w)::value;
        float2 s = make_float2(0.0f, 0.0f);
        if (valid) {
            if (q.kind == 1) {
                float sn, cs;
                sincosf(__ldg(static_cast<const float*>(q.x) + (size_t)b * M + n), &sn, &cs);
                s = make_float2(cs, sn);
            } else {
                s = __ldg(static_cast<const float2*>(q.x) + (size_t)b * M + n);
            }
        }
        v[w] = s;
    });
    row_sync<P::TPR>(slot);
    row_fft<M, false, false, false>(v, buf, t, slot);
    float pt = 0.0f;
    sfor<0, P::VALS>([&](auto w) { pt = fmaf(v[w].x, v[w].x, fmaf(v[w].y, v[w].y, pt)); });
    const float ptot = slot_sum<P::TPR>(pt, red, slot);
    const float inv = ptot > 0.0f ? 1.0f / ptot : 0.0f;
    constexpr float invN = 1.0f / (float)M;
    float d2 = 0.0f;
    sfor<0, P::VALS>([&](auto w) {
        const float d = fmaf(fmaf(v[w].x, v[w].x, v[w].y * v[w].y), inv, -invN);
        d2 = fmaf(d, d, d2);
    });
    const float sv = slot_sum<P::TPR>(d2, red, slot) * invN;
    const float kf = 2.0f * invN * inv;
    const float nsv = (float)M * sv;
    sfor<0, P::VALS>([&](auto w) {
        const float2 x = v[w];
        const float d = fmaf(fmaf(x.x, x.x, x.y * x.y), inv, -invN);
        const float c = kf * (d - nsv);
        v[w] = make_float2(c * x.x, -c * x.y);  // conj(dSV/dP S)
    });
    row_sync<P::TPR>(slot);
    row_fft<M, false, false, false>(v, buf, t, slot);
    if (!valid) return;
    const float wt2 = 2.0f * q.weight;
    sfor<0, P::VALS>([&](auto w) {
        const int n = t + P::TPR * decltype(w)::value;
        const float2 g = make_float2(v[w].x, -v[w].y);  // dSV/ds*[n]
        const size_t i = (size_t)b * M + n;
        if (q.grad_s) {
            float2 o = make_float2(wt2 * g.x, wt2 * g.y);
            if (q.accumulate) o = cadd(o, q.grad_s[i]);
            q.grad_s[i] = o;
        }
        if (q.grad_phi) {
            float2 s;
            if (q.kind == 1) {
                float sn, cs;
                sincosf(static_cast<const float*>(q.x)[i], &sn, &cs);
                s = make_float2(cs, sn);
            } else {
                s = static_cast<const float2*>(q.x)[i];
            }
            float o = wt2 * (g.y * s.x - g.x * s.y);
            if (q.accumulate) o += q.grad_phi[i];
            q.grad_phi[i] = o;
        }
    });
    if (t == 0) {
        if (q.out8) {
            q.out8[(size_t)b * 8] += q.weight * sv;
            q.out8[(size_t)b * 8 + 7] = sv;
        }
        if (q.sv) q.sv[b] = sv;
    }
}

template <int M>
cudaError_t run_spectral_m(const SpecParams& q, cudaStream_t st) {
    using P = RowPlan<M>;
    constexpr int SLOTS = P::THREADS / P::TPR;
    const size_t smem = row_buffer_bytes<M>() + kRedBytes;
    cudaError_t e = cudaFuncSetAttribute(spectral_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((q.B + SLOTS - 1) / SLOTS);
    spectral_kernel<M><<<grid, P::THREADS, smem, st>>>(q);
    return cudaGetLastError();
}

// ---------------------------------------------------------- composite terms
// One row slot per waveform, row length M >= 2N - 1 (no circular wrap):
//   S = DFT_M(s), r[k] = IDFT_M(|S|^2)[k] = sum_n s[n] conj(s[n-k]) (the
//   zero-Doppler column of the AF, lag k at index k mod M),
//   a2 = (|r|^2 + eps) / E^2, W = sum_{|k| < N} |k| sigmoid(gamma (a2 - 1/2)),
//   G[k] = dL/dr*[k] = w_width |k| gamma sig (1 - sig) r[k] / E^2,
//   dL/ds* = IDFT_M(2 Re(DFT_M(G)) S) + energy term + w_const dV/ds*,
// the product rule on r[k] written as a convolution plus a correlation with
// s.  Five transforms per waveform; Re(DFT(G)) waits in shared memory while
// S is transformed again.
template <int M>
__global__ void __launch_bounds__(RowPlan<M>::THREADS, RowPlan<M>::MIN_BLOCKS) composite_kernel(CompParams q) {
    using P = RowPlan<M>;
    constexpr int SLOTS = P::THREADS / P::TPR;
    extern __shared__ __align__(256) unsigned char smem[];
    float2* bufs = reinterpret_cast<float2*>(smem);
    float* stash = reinterpret_cast<float*>(smem + row_buffer_bytes<M>());
    float* red = stash + (size_t)SLOTS * M;
    const int tid = threadIdx.x, slot = tid / P::TPR, t = tid % P::TPR;
    const int b = blockIdx.x * SLOTS + slot;
    const bool valid = b < q.B;  // slot-uniform
    const int N = q.N;
    float2* buf = bufs + (size_t)slot * (P::SPLIT ? P::SMEM_ROW / 2 : P::SMEM_ROW);
    float* st = stash + (size_t)slot * M;
    auto load = [&](float2* v) {
        sfor<0, P::VALS>([&](auto w) {
            const int n = t + P::TPR * decltype(w)::value;
            float2 s = make_float2(0.0f, 0.0f);
            if (valid && n < N) {
                if (q.kind == 1) {
                    float sn, cs;
                    sincosf(__ldg(static_cast<const float*>(q.x) + (size_t)b * N + n), &sn, &cs);
                    s = make_float2(cs, sn);
                } else {
                    s = __ldg(static_cast<const float2*>(q.x) + (size_t)b * N + n);
                }
            }
            v[w] = s;
        });
    };
    float2 v[P::VALS];
    load(v);
    // energy and the modulus statistics
    float e = 0.0f, am = 0.0f;
    sfor<0, P::VALS>([&](auto w) {
        const float a2 = fmaf(v[w].x, v[w].x, v[w].y * v[w].y);
        e += a2;
        am += sqrtf(a2);
    });
    const float E = slot_sum<P::TPR>(e, red, slot);
    const float mu = slot_sum<P::TPR>(am, red, slot) / (float)N;
    float vv = 0.0f;
    sfor<0, P::VALS>([&](auto w) {
        const int n = t + P::TPR * decltype(w)::value;
        const float d = sqrtf(fmaf(v[w].x, v[w].x, v[w].y * v[w].y)) - mu;
        if (n < N) vv = fmaf(d, d, vv);
    });
    const float V = slot_sum<P::TPR>(vv, red, slot) / (float)N;
    // S, then r = conj(DFT(|S|^2)) / M
    row_sync<P::TPR>(slot);
    row_fft<M, false, false, false>(v, buf, t, slot);
    sfor<0, P::VALS>([&](auto w) { v[w] = make_float2(fmaf(v[w].x, v[w].x, v[w].y * v[w].y), 0.0f); });
    row_sync<P::TPR>(slot);
    row_fft<M, false, false, false>(v, buf, t, slot);
    const float invE2 = E > 0.0f ? 1.0f / (E * E) : 0.0f;
    const float invM = 1.0f / (float)M;
    float wsum = 0.0f, esum = 0.0f;
    sfor<0, P::VALS>([&](auto w) {
        const int i = t + P::TPR * decltype(w)::value;
        const int k = i <= M / 2 ? i : i - M;
        const int ak = k < 0 ? -k : k;
        const float2 r = make_float2(v[w].x * invM, -v[w].y * invM);
        float2 g = make_float2(0.0f, 0.0f);
        if (ak < N) {
            const float a2 = fmaf(fmaf(r.x, r.x, r.y * r.y), invE2, q.eps * invE2);
            const float sg = 1.0f / (1.0f + __expf(-q.gamma * (a2 - 0.5f)));
            wsum = fmaf((float)ak, sg, wsum);
            const float d = (float)ak * q.gamma * sg * (1.0f - sg);
            esum = fmaf(d, a2, esum);
            const float c = q.w_width * d * invE2;
            g = make_float2(c * r.x, c * r.y);
        }
        v[w] = g;
    });
    const float W = slot_sum<P::TPR>(wsum, red, slot);
    const float dLdE = -2.0f * q.w_width * slot_sum<P::TPR>(esum, red, slot) / E;
    // Re(DFT(G)) into the stash, S again, then the adjoint of 2 Re(G^) S
    row_sync<P::TPR>(slot);
    row_fft<M, false, false, false>(v, buf, t, slot);
    sfor<0, P::VALS>([&](auto w) { st[t + P::TPR * decltype(w)::value] = 2.0f * v[w].x; });
    load(v);
    row_sync<P::TPR>(slot);
    row_fft<M, false, false, false>(v, buf, t, slot);
    sfor<0, P::VALS>([&](auto w) {
        const float rg = st[t + P::TPR * decltype(w)::value] * invM;
        v[w] = make_float2(rg * v[w].x, -rg * v[w].y);  // conj(y), y = 2 Re(G^) S / M
    });
    row_sync<P::TPR>(slot);
    row_fft<M, false, false, false>(v, buf, t, slot);
    if (!valid) return;
    sfor<0, P::VALS>([&](auto w) {
        const int n = t + P::TPR * decltype(w)::value;
        if (n < N) {
            float2 s;
            if (q.kind == 1) {
                float sn, cs;
                sincosf(static_cast<const float*>(q.x)[(size_t)b * N + n], &sn, &cs);
                s = make_float2(cs, sn);
            } else {
                s = static_cast<const float2*>(q.x)[(size_t)b * N + n];
            }
            const float as = sqrtf(fmaf(s.x, s.x, s.y * s.y));
            const float cv = as > 0.0f ? q.w_const * (as - mu) / ((float)N * as) : 0.0f;
            const float k2 = dLdE + cv;  // real multiplier of s[n]
            const float2 gw = make_float2(fmaf(k2, s.x, v[w].x), fmaf(k2, s.y, -v[w].y));  // dL/ds*[n]
            const size_t i = (size_t)b * N + n;
            if (q.grad_s) {
                float2 o = make_float2(2.0f * gw.x, 2.0f * gw.y);
                if (q.accumulate) o = cadd(o, q.grad_s[i]);
                q.grad_s[i] = o;
            }
            if (q.grad_phi) {
                float o = 2.0f * (gw.y * s.x - gw.x * s.y);
                if (q.accumulate) o += q.grad_phi[i];
                q.grad_phi[i] = o;
            }
        }
    });
    if (t == 0) {
        if (q.out8) q.out8[(size_t)b * 8] += q.w_width * W + q.w_const * V;
        if (q.terms) {
            q.terms[2 * (size_t)b] = W;
            q.terms[2 * (size_t)b + 1] = V;
        }
    }
}

template <int M>
cudaError_t run_composite_m(const CompParams& q, cudaStream_t st) {
    using P = RowPlan<M>;
    constexpr int SLOTS = P::THREADS / P::TPR;
    const size_t smem = row_buffer_bytes<M>() + (size_t)SLOTS * M * sizeof(float) + kRedBytes;
    if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(composite_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((q.B + SLOTS - 1) / SLOTS);
    composite_kernel<M><<<grid, P::THREADS, smem, st>>>(q);
    return cudaGetLastError();
}

// One pass per row: lag product, forward DFT, loss partials and, for rows
// whose weights are uniform over the row, the gradient remainder of the split
// adjoint (see af_backward_kernel) -- no recomputation, no stored AF.
//
// The PSL term needs p - p0 = (exp(beta a2) - 1) / Z with Z = sum_Omega
// exp(beta Ahat^2) unknown until every row is done.  Each row slot keeps a
// running log-sum-exp shift mx (the largest weighted a2 it has seen), forms
// c = w (e - e0) w_psl / E^2 with e = exp(beta (a2 - mx)), e0 = exp(-beta mx),
// and when mx grows rescales what it has accumulated by exp(beta (mx_old -
// mx_new)).  At the end the slots are brought to the CTA's largest shift, and
// the loss finalisation gives each CTA the factor exp(beta (mx_cta -
// PSL_soft)) that turns its partial into the true remainder.  With w_psl = 0
// the remainder is c = (w - w_b) w_isl / E^2, independent of the shift, and
// every row is fused.  No barrier spans the CTA inside the row loop, so the
// slots drift apart and overlap their shared-memory and arithmetic phases.
//
// Rows r_lo..defer_hi (those holding mainlobe-box cells, whose weights are
// not uniform) contribute loss partials only; af_backward_kernel adds their
// gradient once PSL_soft is known.  On the PSL path every slot owns its
// accumulator (acc_copies == slot count).
template <int M, bool HALF, bool RO, int V = 0>
__device__ __forceinline__ void fused_item(const AfParams& p, int b, int tile, unsigned char* smem) {
    const bool phase_only = RO || p.phase_only;  // RO: only dL/dphi is wanted, known at compile time
    using P = RowPlan<M, V>;
    constexpr int SLOTS = P::THREADS / P::TPR;
    constexpr int NW = P::THREADS / 32;
    // the waveform's parameters live in shared memory (CTA-uniform), so they
    // are re-read after barriers instead of occupying registers
    __shared__ Wave s_wave;
    if (threadIdx.x == 0) s_wave = wave_of(p, b);
    __syncthreads();
    const Wave& wv = s_wave;
    float2* s_sm = reinterpret_cast<float2*>(smem);
    float2* bufs = reinterpret_cast<float2*>(smem + smem_signal_bytes<M>(sig_len(p)));
    float2* acc_all = reinterpret_cast<float2*>(smem + smem_signal_bytes<M>(sig_len(p)) + row_buffer_bytes<M, V>());
    float* red = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(acc_all) +
                                          acc_region_bytes(p));
    // red: [0,16) reductions, [32,48) slot-max scratch (TPR > 32), [64, 64+SLOTS) final slot shifts
    // (SLOTS <= 64), [128, 128 + 4 NW) float4s

    const int tid = threadIdx.x, slot = tid / P::TPR, t = tid % P::TPR;
    for (int i = tid; i < (int)(acc_region_bytes(p) / sizeof(float2)); i += P::THREADS)
        acc_all[i] = make_float2(0.0f, 0.0f);
    const float E = load_signal(wv, s_sm, red);  // includes __syncthreads
    // the item's constants live in shared memory and are re-read after each
    // transform, so that none of them occupies a register during the FFTs
    __shared__ float s_k[6];
    if (tid == 0) {
        if (tile == 0) p.out8[(size_t)b * 8 + 4] = E;
        const float invE2 = 1.0f / (E * E);
        const float bl2 = wv.beta * 1.4426950408889634f;  // beta * log2(e)
        s_k[0] = invE2;
        s_k[1] = wv.eps * invE2;   // eps / E^2
        s_k[2] = bl2;
        s_k[3] = wv.w_psl * invE2;  // cP
        s_k[4] = wv.w_isl * invE2;  // cI
        s_k[5] = invE2 * bl2;       // exponent per unit |X|^2
    }
    __syncthreads();
    float2* buf = bufs + (size_t)slot * (P::SPLIT ? P::SMEM_ROW / 2 : P::SMEM_ROW);
    const ColMasks cm = col_masks<M>(wv, t);
    constexpr unsigned long long full_mask = P::VALS == 64 ? ~0ull : ((1ull << P::VALS) - 1ull);
    const int turns = SLOTS / p.acc_copies;
    const int my_turn = slot / p.acc_copies;
    float2* acc = acc_all + (size_t)(slot % p.acc_copies) * acc_stride(wv.N, P::TPR);
    float* acc_r = reinterpret_cast<float*>(acc_all) + (size_t)(slot % p.acc_copies) * acc_stride(wv.N, P::TPR);

    const int row0 = wv.r_lo + tile * wv.rows_per_tile;
    const int row_end = min(row0 + wv.rows_per_tile, wv.r_hi + 1);
    // iterations for the rows this tile actually holds (CTA-uniform)
    const int iters = max(0, row_end - row0 + SLOTS - 1) / SLOTS;

    float isl = 0.0f, zs = 0.0f, ts = 0.0f, cs = 0.0f;
    const bool fixed = wv.lse_fix > 0.0f;      // fixed shift: no running maximum
    float mx = fixed ? wv.lse_fix : -CUDART_INF_F;  // slot-uniform shift (in a2 units)
    float hm = -CUDART_INF_F;  // largest weighted a2 (fixed shift)
    float2 v[P::VALS];
    for (int it = 0; it < iters; ++it) {
        const int k = row0 + slot + it * SLOTS;
        const bool valid = k < row_end;
        const bool grad_row = valid && k > wv.defer_hi && !(phase_only && k == 0);
        // a warp of several row slots none of which holds a valid row skips
        // both transforms; it still runs the scatter below, with nothing to
        // add, so that it joins the CTA's barriers when slots take turns.  Only
        // the last iteration of a tile can hold such warps.  (A slot of whole
        // warps already skips the adjoint of an invalid row.)
        const bool live = P::TPR >= 32 || row0 + (tid >> 5) * (32 / P::TPR) + it * SLOTS < row_end;
        if (live) {
            build_lag_row<M, HALF>(v, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, valid);
            // one transform instance, run twice: the forward DFT, then the adjoint
            // as conj(DFT(conj(c X))) -- the epilogue writes conj(c X) and the
            // scatter reads the conjugated result
#pragma unroll 1
            for (int ph = 0; ph < 2; ++ph) {
                row_sync<P::TPR>(slot);
                row_fft<M, false, false, false, V>(v, buf, t, slot);
                if (ph == 1) break;
                const float invE2 = s_k[0], eps_n = s_k[1], bl2 = s_k[2], cP = s_k[3], cI = s_k[4];
                const bool psl_mode = wv.w_psl != 0.0f;
                const float wb = valid ? (float)base_weight(wv, k) : 0.0f;
                // A row every cell of which carries the same weight (the window
                // spans all Doppler bins, delay k and/or -k in it, no mainlobe-box
                // cell) takes the fast path; the test is slot-uniform.
                const bool in_pos = k >= wv.k_lo && k <= wv.k_hi;
                const bool in_neg = k > 0 && -k >= wv.k_lo && -k <= wv.k_hi;
                if (fixed && valid && wv.full_m && k > wv.k_ml && (in_pos || in_neg)) {
                    // accumulate P = sum |X|^2, Z = sum e, Q = sum e |X|^2 and
                    // apply the weight, 1/E^2 and eps once per row; e = exp(beta
                    // (a2 - mx)) from |X|^2 in one FMA; c = Kp (e - e0) + Ki
                    const float wrow = (in_pos && in_neg) ? 2.0f : 1.0f;
                    const float sh = mx * bl2;
                    const float e0 = ex2a(-sh);
                    const float Kp = (grad_row && psl_mode) ? wrow * cP : 0.0f;
                    const float Ki = (grad_row && !psl_mode) ? (wrow - wb) * cI : 0.0f;
                    const float Kc0 = fmaf(-e0, Kp, Ki);
                    const float kexp = s_k[5], kofs = fmaf(eps_n, bl2, -sh);
                    float rP[2] = {0.0f, 0.0f}, rZ[2] = {0.0f, 0.0f}, rQ[2] = {0.0f, 0.0f};
                    float rH[2] = {0.0f, 0.0f};
                    sfor<0, P::VALS>([&](auto w) {
                        constexpr int h = decltype(w)::value & 1;
                        const float2 x = v[w];
                        const float p2 = fmaf(x.x, x.x, x.y * x.y);
                        const float e = ex2v(fmaf(p2, kexp, kofs));
                        rH[h] = fmaxf(rH[h], p2);
                        rP[h] += p2;
                        rZ[h] += e;
                        rQ[h] = fmaf(e, p2, rQ[h]);
                        const float c = fmaf(e, Kp, Kc0);
                        v[w] = make_float2(c * x.x, -c * x.y);
                    });
                    const float sa2 = fmaf(rP[0] + rP[1], invE2, (float)P::VALS * eps_n);  // sum a2
                    const float Zr = rZ[0] + rZ[1];
                    const float sea2 = fmaf(rQ[0] + rQ[1], invE2, eps_n * Zr);            // sum e a2
                    isl = fmaf(wrow, sa2, isl);
                    zs = fmaf(wrow, Zr, zs);
                    ts = fmaf(wrow, sea2, ts);
                    cs += fmaf(Kp, fmaf(-e0, sa2, sea2), Ki * sa2);
                    hm = fmaxf(hm, fmaf(fmaxf(rH[0], rH[1]), invE2, eps_n));
                } else {
                    const RowMasks rmk = row_masks(wv, cm, k);
                    const bool uniform = !valid || (rmk.one == full_mask && (rmk.two == 0ull || rmk.two == full_mask));
                    const float wrow = valid ? (rmk.two != 0ull ? 2.0f : (rmk.one != 0ull ? 1.0f : 0.0f)) : 0.0f;
                    // registers with weight 0 and no row-uniform part to take out
                    // (wb = 0): their loss terms and their adjoint input c X are
                    // 0.  A narrow Doppler window leaves most registers so, in
                    // the same registers on every lane of a warp, so the branches
                    // below skip the work for the whole warp.
                    const unsigned long long need = !valid ? 0ull : (wb != 0.0f ? full_mask : rmk.one);
                    // pass 1 (running shift only): largest weighted a2 of the row
                    // (two independent chains)
                    float tmx[2] = {-CUDART_INF_F, -CUDART_INF_F};
                    if (!fixed) {
                        sfor<0, P::VALS>([&](auto w) {
                            if (!mbit<decltype(w)::value>(need)) return;
                            const float2 x = v[w];
                            const float a2 = fmaf(fmaf(x.x, x.x, x.y * x.y), invE2, eps_n);
                            const float wt = uniform ? wrow : mweight<decltype(w)::value>(rmk);
                            tmx[w & 1] = fmaxf(tmx[w & 1], wt > 0.0f ? a2 : -CUDART_INF_F);
                        });
                    }
                    const float rmx = fixed ? mx : slot_max<P::TPR>(fmaxf(tmx[0], tmx[1]), red + 32, slot);
                    if (rmx > mx) {  // slot-uniform
                        const float f = ex2a((mx - rmx) * bl2);  // 0 while mx = -inf
                        zs *= f;
                        ts *= f;
                        if (psl_mode) {
                            cs *= f;
                            if (mx > -CUDART_INF_F) {  // the slot owns its accumulator on this path
                                if (phase_only) {
                                    for (int n = t; n < wv.N; n += P::TPR) acc_r[n] *= f;
                                } else {
                                    for (int n = t; n < wv.N; n += P::TPR) {
                                        const float2 a = acc[n];
                                        acc[n] = make_float2(a.x * f, a.y * f);
                                    }
                                }
                            }
                        }
                        mx = rmx;
                    }
                    // pass 2: loss partials and the gradient remainder, v = conj(c X)
                    const float sh = mx * bl2;
                    const float e0 = ex2a(-sh);
                    // row sums in two independent chains each (even / odd registers)
                    float r_isl[2] = {0.0f, 0.0f}, r_z[2] = {0.0f, 0.0f}, r_t[2] = {0.0f, 0.0f};
                    float r_c[2] = {0.0f, 0.0f}, r_h[2] = {-CUDART_INF_F, -CUDART_INF_F};
                    sfor<0, P::VALS>([&](auto w) {
                        constexpr int h = decltype(w)::value & 1;
                        if (!mbit<decltype(w)::value>(need)) {
                            v[w] = make_float2(0.0f, 0.0f);
                            return;
                        }
                        const float2 x = v[w];
                        const float a2 = fmaf(fmaf(x.x, x.x, x.y * x.y), invE2, eps_n);
                        const float wt = uniform ? wrow : mweight<decltype(w)::value>(rmk);
                        const float e = wt > 0.0f ? ex2a(fmaf(a2, bl2, -sh)) : 0.0f;
                        r_h[h] = fmaxf(r_h[h], wt > 0.0f ? a2 : -CUDART_INF_F);
                        const float we = wt * e;
                        r_isl[h] = fmaf(wt, a2, r_isl[h]);
                        r_z[h] += we;
                        r_t[h] = fmaf(we, a2, r_t[h]);
                        float c = 0.0f;
                        if (grad_row) c = psl_mode ? wt * (e - e0) * cP : (wt - wb) * cI;
                        r_c[h] = fmaf(c, a2, r_c[h]);
                        v[w] = make_float2(c * x.x, -c * x.y);
                    });
                    isl += r_isl[0] + r_isl[1];
                    zs += r_z[0] + r_z[1];
                    ts += r_t[0] + r_t[1];
                    cs += r_c[0] + r_c[1];
                    hm = fmaxf(hm, fmaxf(r_h[0], r_h[1]));
                }
                if constexpr (P::TPR >= 32) {
                    if (!grad_row) break;  // slot-uniform: the slot is one or more whole warps
                }
            }
        }
        if (phase_only) {
            scatter_row_real<M, HALF>(v, acc_r, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, grad_row, slot, turns,
                                      my_turn, wv.periodic != 0);
        } else if constexpr (!RO) {
            scatter_row<M, HALF, true>(v, acc, s_sm, wv.N, wv.periodic ? k - wv.N : k, t, grad_row, slot, turns,
                                       my_turn, wv.periodic != 0);
        }
    }
    // bring every slot to the CTA's largest shift (fixed shift: the CTA's
    // largest weighted a2, the record's hard maximum)
    float cmx = fixed ? hm : mx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cmx = fmaxf(cmx, __shfl_xor_sync(0xffffffffu, cmx, o));
    if ((tid & 31) == 0) red[tid >> 5] = cmx;
    __syncthreads();
    cmx = red[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) cmx = fmaxf(cmx, red[w]);
    __syncthreads();
    const float fs = fixed ? 1.0f : (mx > -CUDART_INF_F) ? ex2a((mx - cmx) * s_k[2]) : 0.0f;
    zs *= fs;
    ts *= fs;
    if (wv.w_psl != 0.0f && !fixed) {
        cs *= fs;
        if (phase_only) {
            for (int n = t; n < wv.N; n += P::TPR) acc_r[n] *= fs;
        } else {
            for (int n = t; n < wv.N; n += P::TPR) {
                const float2 a = acc[n];
                acc[n] = make_float2(a.x * fs, a.y * fs);
            }
        }
    }
    // loss record {ISL, mx, sum e, sum e a2}, all relative to the CTA shift
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        isl += __shfl_xor_sync(0xffffffffu, isl, o);
        zs += __shfl_xor_sync(0xffffffffu, zs, o);
        ts += __shfl_xor_sync(0xffffffffu, ts, o);
    }
    float4* wred = reinterpret_cast<float4*>(red + 128);
    if ((tid & 31) == 0) wred[tid >> 5] = make_float4(isl, cmx, zs, ts);
    __syncthreads();
    if (tid == 0) {
        float4 a = wred[0];
        for (int w = 1; w < NW; ++w) {
            a.x += wred[w].x;
            a.z += wred[w].z;
            a.w += wred[w].w;
        }
        p.rec[wv.rec_off + tile] = a;
    }
    write_grad_partial<M, V>(p, wv, acc_all, red, cs, tile);
}

template <int M, bool HALF, bool RO, int V = 0>
__global__ void __launch_bounds__(RowPlan<M, V>::THREADS, RowPlan<M, V>::MIN_BLOCKS) af_fused_kernel(AfParams p) {
    extern __shared__ __align__(256) unsigned char smem[];
    for_each_item(p, [&](int b, int tile) { fused_item<M, HALF, RO, V>(p, b, tile, smem); });
}

// ---------------------------------------------------------- host launchers
template <int M, int V = 0, class K>
static cudaError_t launch_rows(K kernel, size_t smem, const AfParams& p, cudaStream_t st) {
    using P = RowPlan<M, V>;
    if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    long long grid = (long long)p.B * p.tiles;
    if (p.items) {  // persistent: as many CTAs as fit on the SMs at once
        const int sms = device_sm_count();
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, P::THREADS, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        const long long cap = (long long)sms * per_sm;
        grid = p.n_items < cap ? p.n_items : cap;
        if (grid < 1) return cudaSuccess;
    }
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kernel<<<(unsigned)grid, P::THREADS, smem, st>>>(p);
    return cudaGetLastError();
}

template <int M>
cudaError_t run_forward_m(const AfParams& p, cudaStream_t st) {
    const size_t smem = forward_smem<M>(sig_len(p));
    if (2 * p.N <= M) return launch_rows<M>(af_forward_kernel<M, true>, smem, p, st);
    return launch_rows<M>(af_forward_kernel<M, false>, smem, p, st);
}
template <int M>
cudaError_t run_loss_m(const AfParams& p, cudaStream_t st) {
    const size_t smem = forward_smem<M>(sig_len(p));
    if (2 * p.N <= M) return launch_rows<M>(af_loss_kernel<M, true>, smem, p, st);
    return launch_rows<M>(af_loss_kernel<M, false>, smem, p, st);
}
template <int M>
cudaError_t run_backward_m(const AfParams& p, cudaStream_t st) {
    if (p.acc_copies < 1 || (RowPlan<M>::THREADS / RowPlan<M>::TPR) % p.acc_copies) return cudaErrorInvalidConfiguration;
    const size_t smem = backward_smem<M>(p.N, p.acc_copies, p.phase_only, p.periodic);
    // the phase-gradient-only kernel carries no complex scatter
    if (p.phase_only) return launch_rows<M>(af_backward_kernel<M, false, true>, smem, p, st);
    return launch_rows<M>(af_backward_kernel<M, false, false>, smem, p, st);
}

// The kernels that run two transforms per row use one transform instance for
// both, so that transform prunes neither a half-zero input nor a half-needed
// output (one inlined transform keeps the register allocation free of
// spills); with N <= M/2 the fused kernel still skips the zero half in the
// lag product and in the scatter.
template <int M>
cudaError_t run_match_m(const AfParams& p, cudaStream_t st) {
    if (p.acc_copies < 1 || (RowPlan<M>::THREADS / RowPlan<M>::TPR) % p.acc_copies) return cudaErrorInvalidConfiguration;
    const size_t smem = backward_smem<M>(p.N, p.acc_copies, p.phase_only, p.periodic);
    if (2 * p.N <= M && !p.periodic) return launch_rows<M>(af_match_kernel<M, true>, smem, p, st);
    return launch_rows<M>(af_match_kernel<M, false>, smem, p, st);
}

template <int M>
cudaError_t run_fused_m(const AfParams& p, cudaStream_t st) {
    if (p.acc_copies < 1 || (RowPlan<M>::THREADS / RowPlan<M>::TPR) % p.acc_copies) return cudaErrorInvalidConfiguration;
    if constexpr (M == 8192) {
        // two row slots per CTA, each with a whole exchange buffer (no
        // real/imaginary split), when the signal is short enough for both to
        // fit: one gradient accumulator per slot, else one shared in turns
        if (2 * p.N <= M && p.phase_only && !p.periodic) {
            for (int a = 2; a >= 1; a /= 2) {
                const size_t smem2 = backward_smem<M, 1>(p.N, a, 1, 0);
                if (smem2 <= kMaxSmem) {
                    AfParams q = p;
                    q.acc_copies = a;
                    return launch_rows<M, 1>(af_fused_kernel<M, true, true, 1>, smem2, q, st);
                }
            }
        }
    }
    const size_t smem = backward_smem<M>(p.N, p.acc_copies, p.phase_only, p.periodic);
    // the phase-gradient-only kernel carries no complex scatter
    if (2 * p.N <= M && p.phase_only) return launch_rows<M>(af_fused_kernel<M, true, true>, smem, p, st);
    if (p.phase_only) return launch_rows<M>(af_fused_kernel<M, false, true>, smem, p, st);
    if (2 * p.N <= M) return launch_rows<M>(af_fused_kernel<M, true, false>, smem, p, st);
    return launch_rows<M>(af_fused_kernel<M, false, false>, smem, p, st);
}

}  // namespace graf

#define GRAF_INSTANTIATE_M(M)                                                      \
    template cudaError_t graf::run_forward_m<M>(const graf::AfParams&, cudaStream_t);  \
    template cudaError_t graf::run_loss_m<M>(const graf::AfParams&, cudaStream_t);     \
    template cudaError_t graf::run_backward_m<M>(const graf::AfParams&, cudaStream_t); \
    template cudaError_t graf::run_fused_m<M>(const graf::AfParams&, cudaStream_t);    \
    template cudaError_t graf::run_spectral_m<M>(const graf::SpecParams&, cudaStream_t);   \
    template cudaError_t graf::run_composite_m<M>(const graf::CompParams&, cudaStream_t);   \
    template cudaError_t graf::run_match_m<M>(const graf::AfParams&, cudaStream_t);
