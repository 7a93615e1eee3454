// graf_af.cu - reductions that follow the row kernels (loss finalisation,
// gradient reduction) and the dispatch over the row length M.
#include <climits>

#include <math_constants.h>

#include "graf.h"
#include "graf_kernels.cuh"

namespace graf {

// The device error word of this device (GRAF_DEVERR_* bits), raised by the
// finalisation kernels and taken (read and cleared in one atomic exchange) by
// graf_get_device_error_word.
__device__ unsigned int g_device_error;
__device__ unsigned int g_device_error_taken;

__global__ void take_device_error_kernel() { g_device_error_taken = atomicExch(&g_device_error, 0u); }

// Device address of this device's error word in the current context (looked
// up at every call: a reset or another context moves it); nullptr on error.
unsigned int* device_error_word_address() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    return static_cast<unsigned int*>(p);
}

int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
        return sms;
    cudaGetLastError();  // no device: clear the error the failed query recorded
    return 152;
}

// |Omega| = |window| - |window intersect mainlobe box|, exact in int64.
__device__ __forceinline__ long long omega_count(const Wave& p) {
    const long long nk = p.k_hi - p.k_lo + 1, nm = p.m_hi - p.m_lo + 1;
    long long bk = 0, bm = 0;
    if (p.k_ml >= 0 && p.m_ml >= 0) {
        const int kl = max(p.k_lo, -p.k_ml), kh = min(p.k_hi, p.k_ml);
        const int ml = max(p.m_lo, -p.m_ml), mh = min(p.m_hi, p.m_ml);
        bk = kh >= kl ? kh - kl + 1 : 0;
        bm = mh >= ml ? mh - ml + 1 : 0;
    }
    return nk * nm - bk * bm;
}

// Hard PSL (beta = +inf): merge the tile records {ISL, max, row, code} --
// ISL in a fixed order, the arg-max by the larger value, then the smaller row,
// then the smaller code -- into out8 = {w_peak max + w_isl ISL, max, ISL, max,
// E, |Omega|, max, 0} (max is PSL_hard, and the limit of PSL_soft and of the
// softmax-weighted mean S_p) and the waveform's peak record.
__device__ void finalize_hard(const AfParams& p, const Wave& wv, int b, int lane, float* out8) {
    double isl = 0.0;
    float bv = -CUDART_INF_F;
    int brow = INT_MAX, bcode = INT_MAX;
    auto better = [](float v, int r, int c, float v2, int r2, int c2) {
        return v > v2 || (v == v2 && (r < r2 || (r == r2 && c < c2)));
    };
    for (int i = lane; i < wv.tiles; i += 32) {
        const float4 r = p.rec[wv.rec_off + i];
        isl += r.x;
        const int rr = __float_as_int(r.z), rc = __float_as_int(r.w);
        if (r.y > -CUDART_INF_F && better(r.y, rr, rc, bv, brow, bcode)) {
            bv = r.y;
            brow = rr;
            bcode = rc;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        isl += __shfl_xor_sync(0xffffffffu, isl, o);
        const float v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const int r2 = __shfl_xor_sync(0xffffffffu, brow, o), c2 = __shfl_xor_sync(0xffffffffu, bcode, o);
        if (better(v2, r2, c2, bv, brow, bcode)) {
            bv = v2;
            brow = r2;
            bcode = c2;
        }
    }
    if (lane == 0) {
        float* o = out8 + (size_t)b * 8;
        const bool any = bv > -CUDART_INF_F;
        const float h = any ? bv : 0.0f;
        o[0] = any ? (float)((double)wv.w_peak * h + (double)wv.w_isl * isl) : 0.0f;
        o[1] = h;
        o[2] = any ? (float)isl : 0.0f;
        o[3] = h;
        o[5] = (float)omega_count(wv);
        o[6] = h;
        o[7] = 0.0f;
        const float E = o[4];
        unsigned int bits = 0;
        if (!(E > 0.0f) || !isfinite(E)) bits |= GRAF_DEVERR_ENERGY;
        if (!isfinite(o[0]) || !isfinite(o[2]) || !isfinite(o[3])) bits |= GRAF_DEVERR_NONFINITE;
        if (bits) atomicOr(&g_device_error, bits);
        if (p.peak) p.peak[b] = make_int4(any ? brow : -1, any ? bcode : 0, __float_as_int(h), 0);
    }
    // every partial of the fused kernel is final (its soft PSL weight is 0)
    if (p.scale)
        for (int i = lane; i < wv.tiles; i += 32) p.scale[wv.rec_off + i] = 1.0f;
}

// One warp per waveform: merge the tile records in a fixed order (double).
__global__ void loss_finalize_kernel(AfParams p, float* out8) {
    const int b = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (b >= p.B) return;
    const Wave wv = wave_of(p, b);
    if (wv.hard) {
        finalize_hard(p, wv, b, lane, out8);
        return;
    }
    const double beta = wv.beta;
    const bool fixed = wv.lse_fix > 0.0f;
    double isl = 0.0, mx = -CUDART_INF, z = 0.0, T = 0.0, hard = -CUDART_INF;
    for (int i = lane; i < wv.tiles; i += 32) {
        const float4 r = p.rec[wv.rec_off + i];
        isl += r.x;
        hard = fmax(hard, (double)r.y);
        if (r.y > -CUDART_INF_F) {
            const double m2 = fixed ? (double)wv.lse_fix : (double)r.y;
            if (m2 > mx) {
                const double f = exp(beta * (mx - m2));
                z = z * f + r.z;
                T = T * f + r.w;
                mx = m2;
            } else {
                const double f = exp(beta * (m2 - mx));
                z += r.z * f;
                T += r.w * f;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double i2 = __shfl_xor_sync(0xffffffffu, isl, o);
        const double m2 = __shfl_xor_sync(0xffffffffu, mx, o);
        const double z2 = __shfl_xor_sync(0xffffffffu, z, o);
        const double t2 = __shfl_xor_sync(0xffffffffu, T, o);
        hard = fmax(hard, __shfl_xor_sync(0xffffffffu, hard, o));
        isl += i2;
        if (m2 > mx) {
            const double f = exp(beta * (mx - m2));
            z = z * f + z2;
            T = T * f + t2;
            mx = m2;
        } else if (m2 > -CUDART_INF) {
            const double f = exp(beta * (m2 - mx));
            z += z2 * f;
            T += t2 * f;
        }
    }
    double psl_soft = 0.0;
    if (lane == 0) {
        float* o = out8 + (size_t)b * 8;
        const double cnt = (double)omega_count(wv);
        if (mx == -CUDART_INF || z <= 0.0) {
            o[0] = 0.0f; o[1] = 0.0f; o[2] = 0.0f; o[3] = 0.0f; o[6] = 0.0f;
        } else {
            psl_soft = mx + log(z) / beta;
            o[0] = (float)(wv.w_psl * psl_soft + wv.w_isl * isl);
            o[1] = (float)psl_soft;
            o[2] = (float)isl;
            o[3] = (float)hard;
            o[6] = (float)(T / z);
        }
        o[5] = (float)cnt;
        o[7] = 0.0f;
        // E was written by the row kernels earlier on this stream
        const float E = o[4];
        unsigned int bits = 0;
        if (!(E > 0.0f) || !isfinite(E)) bits |= GRAF_DEVERR_ENERGY;
        if (!isfinite(o[0]) || !isfinite(o[1]) || !isfinite(o[2]) || !isfinite(o[3])) bits |= GRAF_DEVERR_NONFINITE;
        if (bits) atomicOr(&g_device_error, bits);
    }
    // fused loss + gradient: per-CTA factor that turns a partial accumulated
    // with the CTA's shift mx_cta into the true remainder, exp(beta (mx_cta -
    // PSL_soft)) on the PSL path, 1 on the ISL-only path
    if (p.scale) {
        psl_soft = __shfl_sync(0xffffffffu, psl_soft, 0);
        for (int i = lane; i < wv.tiles; i += 32) {
            const float m = fixed ? wv.lse_fix : p.rec[wv.rec_off + i].y;
            float f = 1.0f;
            if (wv.w_psl != 0.0f && !wv.unscaled)
                f = m > -CUDART_INF_F ? (float)exp(beta * ((double)m - psl_soft)) : 0.0f;
            p.scale[wv.rec_off + i] = f;
        }
    }
}

// s[n] as the row kernels see it (conjugated for the +j periodic AF).
__device__ __forceinline__ float2 signal_at(const Wave& wv, int n) {
    float2 v;
    if (wv.kind == 1) {
        float sn, cs;
        sincosf(static_cast<const float*>(wv.x)[n], &sn, &cs);
        v = make_float2(cs, sn);
    } else {
        v = static_cast<const float2*>(wv.x)[n];
    }
    if (wv.pconj) v.y = -v.y;
    return v;
}

// n +- k wrapped into [0, N) for the periodic AF; -1 where the aperiodic
// lag product has no such sample.
__device__ __forceinline__ int lag_index(const Wave& wv, int i) {
    if (wv.periodic) return i < 0 ? i + wv.N : (i >= wv.N ? i - wv.N : i);
    return (i < 0 || i >= wv.N) ? -1 : i;
}

// dL/ds* of the FFT part: scaled sum of the per-CTA partials of the first
// set (g1) and the unscaled second set (deferred rows, g2), each in a fixed
// order; the same for the per-CTA sums of c a2.
__device__ __forceinline__ void sum_partials(const AfParams& p, const Wave& wv, int b, int n, float2& g1s,
                                             float2& g2s, double* cs) {
    const float2* g1 = p.gpart + wv.gpart_off + n;
    float2 g = make_float2(0.0f, 0.0f);
    double c = 0.0;
    for (int i = 0; i < wv.tiles; ++i) {
        const float f = p.scale ? p.scale[wv.rec_off + i] : 1.0f;
        const float2 a = g1[(size_t)i * wv.N];
        g.x = fmaf(f, a.x, g.x);
        g.y = fmaf(f, a.y, g.y);
        if (cs) c += (double)f * p.csum[wv.rec_off + i];
    }
    g1s = g;
    g = make_float2(0.0f, 0.0f);
    if (p.gpart2) {
        const float2* g2 = p.gpart2 + (size_t)b * p.tiles2 * p.N + n;
        for (int i = 0; i < p.tiles2; ++i) {
            g = cadd(g, g2[(size_t)i * p.N]);
            if (cs) c += p.csum2[(size_t)b * p.tiles2 + i];
        }
    }
    g2s = g;
    if (cs) *cs = c;
}

// grad_phi = 2 Im(dL/ds* conj(s)): the row-uniform part and the energy terms
// are s[n] times real numbers and contribute nothing to it.  In phase-only
// mode the first set already holds Im(dL/ds* conj(s)) (real accumulators);
// the second set (deferred rows) is always complex.
__global__ void grad_phi_kernel(AfParams p, const float* dL, float* grad_phi) {
    const int nblk = (p.N + blockDim.x - 1) / blockDim.x;
    const int b = blockIdx.x / nblk;
    const int n = (blockIdx.x % nblk) * blockDim.x + threadIdx.x;
    const Wave wv = wave_of(p, b);
    if (n >= wv.N) return;
    float2 g1, g2;
    sum_partials(p, wv, b, n, g1, g2, nullptr);
    const float2 s = signal_at(wv, n);
    const float scale = 2.0f * (dL ? dL[b] : 1.0f);
    float im;
    if (p.phase_only) im = g1.x + (g2.y * s.x - g2.x * s.y);
    else im = (g1.y + g2.y) * s.x - (g1.x + g2.x) * s.y;
    // +j periodic AF: the kernels saw conj(s) = exp(-j phi), so dL/dphi flips sign
    const float val = wv.pconj ? -scale * im : scale * im;
    grad_phi[wv.out_off + n] = p.grad_acc ? grad_phi[wv.out_off + n] + val : val;
}

// Per waveform, in FP64: U = sum_k w_b(k) (C[k] + eps) over the transformed
// rows, C[k] = sum_n |s[n]|^2 |s[n-k]|^2 (Parseval: sum_m |X[k,m]|^2 = M C[k]),
// and E = sum_n |s[n]|^2 -> usum[2b], usum[2b+1].
__global__ void uniform_sum_kernel(AfParams p) {
    extern __shared__ double a_sm[];
    __shared__ double red[32];
    const int b = blockIdx.x;
    const Wave wv = wave_of(p, b);
    for (int n = threadIdx.x; n < wv.N; n += blockDim.x) {
        const float2 s = signal_at(wv, n);
        a_sm[n] = (double)s.x * s.x + (double)s.y * s.y;
    }
    __syncthreads();
    double acc = 0.0;
    for (int k = wv.r_lo + threadIdx.x; k <= wv.r_hi; k += blockDim.x) {
        const int wb = base_weight(wv, k);
        if (wb == 0) continue;
        double c = 0.0;
        for (int n = 0; n < wv.N; ++n) {
            const int j = lag_index(wv, n - k);
            if (j >= 0) c += a_sm[n] * a_sm[j];
        }
        acc += wb * (c + (double)wv.eps);
    }
    // E in FP64 from the same |s|^2, so the closed form cancels exactly
    double e = 0.0;
    for (int n = threadIdx.x; n < wv.N; n += blockDim.x) e += a_sm[n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = acc;
        red[16 + (threadIdx.x >> 5)] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, es = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
            s += red[w];
            es += red[16 + w];
        }
        p.usum[2 * b] = s;
        p.usum[2 * b + 1] = es;
    }
}

// grad_s = 2 dL [g_fft + dLdE_fft s + g_u], with (all FP64 after the sums)
//   dLdE_fft = -2 E sum_tiles csum           (energy term of the FFT part)
//   g_u[n]   = A' M s[n] ( sum_k w_b(k)(|s[n-k]|^2 [n>=k] + |s[n+k]|^2 [n+k<N]) / E^2
//                          - 2 U / E^3 )    (row-uniform part in closed form)
// with A' = w_isl + w_psl p0, p0 = exp(-beta PSL_soft) evaluated exactly as in
// the backward kernel.  grad_phi, if requested, uses g_fft alone.
__global__ void grad_s_kernel(AfParams p, const float* dL, float2* grad_s, float* grad_phi) {
    extern __shared__ double a_sm[];
    const int nblk = (p.N + blockDim.x - 1) / blockDim.x;
    const int b = blockIdx.x / nblk;
    const int n0 = (blockIdx.x % nblk) * blockDim.x;
    const Wave wv = wave_of(p, b);
    for (int n = threadIdx.x; n < wv.N; n += blockDim.x) {
        const float2 s = signal_at(wv, n);
        a_sm[n] = (double)s.x * s.x + (double)s.y * s.y;
    }
    __syncthreads();
    const int n = n0 + threadIdx.x;
    if (n >= wv.N) return;
    double cs = 0.0;
    float2 g1, g2;
    sum_partials(p, wv, b, n, g1, g2, &cs);
    const float2 g = cadd(g1, g2);
    const float2 s = signal_at(wv, n);
    const float psl_soft = p.saved8 ? p.saved8[(size_t)b * 8 + 1] : 0.0f;
    const double E = p.usum[2 * b + 1];
    const float bl2 = wv.beta * 1.4426950408889634f;
    const float p0 = ex2a(-(psl_soft * bl2));
    const double Ap = (double)fmaf(wv.w_psl, p0, wv.w_isl);
    double corr = 0.0;
    for (int k = wv.r_lo; k <= wv.r_hi; ++k) {
        const int wb = base_weight(wv, k);
        if (wb == 0) continue;
        double t = 0.0;
        const int j1 = lag_index(wv, n - k), j2 = lag_index(wv, n + k);
        if (j1 >= 0) t += a_sm[j1];
        if (j2 >= 0) t += a_sm[j2];
        corr += wb * t;
    }
    const double gu = Ap * (double)wv.M * (corr / (E * E) - 2.0 * p.usum[2 * b] / (E * E * E));
    // origin cell, left out of the FFT part: its exact total is -2 eps c00 s / E
    double c00 = 0.0;
    if (wv.k_lo <= 0 && wv.k_hi >= 0 && wv.m_lo <= 0 && wv.m_hi >= 0) {
        const int w00 = (wv.k_ml >= 0 && wv.m_ml >= 0) ? 0 : 1;
        const double a00 = 1.0 + (double)wv.eps / (E * E);
        const double pr = exp((double)wv.beta * (a00 - (double)psl_soft));
        c00 = ((w00 - base_weight(wv, 0)) * Ap + (w00 > 0 ? w00 * (double)wv.w_psl * (pr - (double)p0) : 0.0)) /
              (E * E);
    }
    const double coef = -2.0 * E * cs + gu - 2.0 * (double)wv.eps * c00 / E;  // real multiplier of s[n]
    const double scale = 2.0 * (dL ? (double)dL[b] : 1.0);
    // +j periodic AF: everything above is the gradient with respect to u =
    // conj(s); the gradient with respect to s is its conjugate, and dL/dphi
    // flips sign
    const float cj = wv.pconj ? -1.0f : 1.0f;
    float2 gv = make_float2((float)(scale * (g.x + coef * s.x)), cj * (float)(scale * (g.y + coef * s.y)));
    if (p.grad_acc) gv = cadd(gv, grad_s[wv.out_off + n]);
    grad_s[wv.out_off + n] = gv;
    if (grad_phi) {
        const float pv = cj * (float)(scale * ((double)g.y * s.x - (double)g.x * s.y));
        grad_phi[wv.out_off + n] = p.grad_acc ? grad_phi[wv.out_off + n] + pv : pv;
    }
}

// e^{-2 pi j q n / M} for M a power of two: the exponent reduced exactly in
// integers, then sincospi of a value in [0, 2).
__device__ __forceinline__ float2 twiddle_qn(int q, int n, int M) {
    const int r = (int)(((unsigned)q * (unsigned)n) & (unsigned)(M - 1));
    float sn, cs;
    sincospif(2.0f * (float)r / (float)M, &sn, &cs);
    return make_float2(cs, -sn);
}

// X[k, q] = sum_n u[n] conj(u[n - k]) e^{-2 pi j q n / M} of transformed row
// k >= 0 (lag k - N over the doubled signal for the periodic AF), summed by
// the CTA in a fixed order; every thread gets the result.  `red` holds 2
// floats per warp.
__device__ float2 row_bin(const Wave& wv, const float2* u, int k, int q, float* red) {
    float2 acc = make_float2(0.0f, 0.0f);
    const int n0 = wv.periodic ? 0 : k;
    for (int n = n0 + (int)threadIdx.x; n < wv.N; n += (int)blockDim.x) {
        const int j = wv.periodic ? ((n - k) & (wv.N - 1)) : n - k;
        const float2 r = cmulc(u[n], u[j]);
        const float2 w = twiddle_qn(q, n, wv.M);
        acc = make_float2(fmaf(r.x, w.x, fmaf(-r.y, w.y, acc.x)), fmaf(r.x, w.y, fmaf(r.y, w.x, acc.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[2 * (threadIdx.x >> 5)] = acc.x;
        red[2 * (threadIdx.x >> 5) + 1] = acc.y;
    }
    __syncthreads();
    float2 x = make_float2(0.0f, 0.0f);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x = make_float2(x.x + red[2 * w], x.y + red[2 * w + 1]);
    return x;
}

// Hard PSL gradient: per waveform, w_peak dAhat^2/du* at the arg-max cell
// (k, q) of its peak record -- one delay row, in closed form (the product rule
// on the one sum X = sum_n u[n] conj(u[n-k]) W^(q n), W = e^{-2 pi j / M}):
//   dAhat^2/du*[p] = (X u[p-k] conj(W^(q p)) + conj(X) u[p+k] W^(q (p+k))) / E^2
//                    - 2 Ahat^2 u[p] / E,
// a term absent where p - k or p + k leaves [0, N) (taken mod N for the
// periodic AF).  u = s, or conj(s) for the +j periodic AF (mapped back as in
// grad_s_kernel).
__global__ void peak_grad_kernel(AfParams p, const float* dL, float2* grad_s, float* grad_phi, int accumulate) {
    extern __shared__ float2 u_sm[];
    __shared__ float red[64];
    __shared__ double dred[32];
    const int b = blockIdx.x;
    const Wave wv = wave_of(p, b);
    const int N = wv.N, M = wv.M;
    double e = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const float2 v = signal_at(wv, n);
        u_sm[n] = v;
        e += (double)v.x * v.x + (double)v.y * v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) dred[threadIdx.x >> 5] = e;
    __syncthreads();
    double E = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) E += dred[w];
    const int4 pk = p.peak[b];
    const int k = pk.x, q = pk.y;
    // nothing to add: Omega empty, no weight, or row 0 of a unit-modulus
    // phase code (|s[n]|^2 = 1 whatever the phases)
    const bool none = k < 0 || q < 0 || wv.w_peak == 0.0f || (wv.kind == 1 && k == 0);
    float2 X = make_float2(0.0f, 0.0f);
    if (!none) X = row_bin(wv, u_sm, k, q, red);
    const double invE2 = 1.0 / (E * E);
    const double a2 = ((double)X.x * X.x + (double)X.y * X.y + (double)wv.eps) * invE2;
    const float scale = 2.0f * wv.w_peak * (dL ? dL[b] : 1.0f);
    const float cj = wv.pconj ? -1.0f : 1.0f;
    const bool add = !none;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float2 g = make_float2(0.0f, 0.0f);
        if (add) {
            const float2 un = u_sm[n];
            const int jm = wv.periodic ? ((n - k) & (N - 1)) : n - k;  // p - k
            const int jp = wv.periodic ? ((n + k) & (N - 1)) : n + k;  // p + k
            float2 d = make_float2(0.0f, 0.0f);
            if (jm >= 0) {  // X u[p-k] conj(W^(q p))
                const float2 w = twiddle_qn(q, n, M);
                d = cadd(d, cmulc(cmul(X, u_sm[jm]), w));
            }
            if (jp < N) {  // conj(X) u[p+k] W^(q (p+k))
                const float2 w = twiddle_qn(q, wv.periodic ? jp : n + k, M);
                d = cadd(d, cmul(cmulc(u_sm[jp], X), w));
            }
            const float c1 = (float)invE2, c2 = (float)(2.0 * a2 / E);
            g = make_float2(fmaf(c1, d.x, -c2 * un.x), fmaf(c1, d.y, -c2 * un.y));  // dAhat^2/du*
            if (grad_phi) {
                const float pv = cj * scale * (g.y * un.x - g.x * un.y);
                grad_phi[wv.out_off + n] = accumulate ? grad_phi[wv.out_off + n] + pv : pv;
            }
            if (grad_s) {
                float2 gv = make_float2(scale * g.x, cj * scale * g.y);
                if (accumulate) gv = cadd(gv, grad_s[wv.out_off + n]);
                grad_s[wv.out_off + n] = gv;
            }
        } else if (!accumulate) {
            if (grad_phi) grad_phi[wv.out_off + n] = 0.0f;
            if (grad_s) grad_s[wv.out_off + n] = make_float2(0.0f, 0.0f);
        }
    }
}

// Per-waveform match loss: the tile partials summed in order.
__global__ void match_finalize_kernel(AfParams p, float* loss_out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.B) return;
    const Wave wv = wave_of(p, b);
    double s = 0.0;
    for (int i = 0; i < wv.tiles; ++i) s += p.mpart[wv.rec_off + i];
    if (loss_out) loss_out[b] = (float)s;
    if (p.out8) p.out8[(size_t)b * 8] += (float)((double)p.match_w * s);
    if (!isfinite(s)) atomicOr(&g_device_error, GRAF_DEVERR_NONFINITE);
}

#define GRAF_DISPATCH_M(FN, M, ...)                      \
    switch (M) {                                         \
        case 8: return FN<8>(__VA_ARGS__);               \
        case 16: return FN<16>(__VA_ARGS__);             \
        case 32: return FN<32>(__VA_ARGS__);             \
        case 64: return FN<64>(__VA_ARGS__);             \
        case 128: return FN<128>(__VA_ARGS__);           \
        case 256: return FN<256>(__VA_ARGS__);           \
        case 512: return FN<512>(__VA_ARGS__);           \
        case 1024: return FN<1024>(__VA_ARGS__);         \
        case 2048: return FN<2048>(__VA_ARGS__);         \
        case 4096: return FN<4096>(__VA_ARGS__);         \
        case 8192: return FN<8192>(__VA_ARGS__);         \
        case 16384: return FN<16384>(__VA_ARGS__);       \
        default: return cudaErrorInvalidValue;           \
    }

template <int M>
static size_t smem_need_m(int N, int which) {
    if (which == 2) {
        const int a = backward_acc_copies<M>(N);
        return a ? backward_smem<M>(N, a) : (size_t)-1;
    }
    return forward_smem<M>(N);
}
static size_t smem_need(int M, int N, int which) {
    switch (M) {
        case 8: return smem_need_m<8>(N, which);
        case 16: return smem_need_m<16>(N, which);
        case 32: return smem_need_m<32>(N, which);
        case 64: return smem_need_m<64>(N, which);
        case 128: return smem_need_m<128>(N, which);
        case 256: return smem_need_m<256>(N, which);
        case 512: return smem_need_m<512>(N, which);
        case 1024: return smem_need_m<1024>(N, which);
        case 2048: return smem_need_m<2048>(N, which);
        case 4096: return smem_need_m<4096>(N, which);
        case 8192: return smem_need_m<8192>(N, which);
        case 16384: return smem_need_m<16384>(N, which);
        default: return (size_t)-1;
    }
}

size_t row_kernel_smem(int M, int N, int which) { return smem_need(M, N, which); }

int acc_copies_for(int M, int N, int real, int per) {
    switch (M) {
        case 8: return backward_acc_copies<8>(N, real, per);
        case 16: return backward_acc_copies<16>(N, real, per);
        case 32: return backward_acc_copies<32>(N, real, per);
        case 64: return backward_acc_copies<64>(N, real, per);
        case 128: return backward_acc_copies<128>(N, real, per);
        case 256: return backward_acc_copies<256>(N, real, per);
        case 512: return backward_acc_copies<512>(N, real, per);
        case 1024: return backward_acc_copies<1024>(N, real, per);
        case 2048: return backward_acc_copies<2048>(N, real, per);
        case 4096: return backward_acc_copies<4096>(N, real, per);
        case 8192: return backward_acc_copies<8192>(N, real, per);
        case 16384: return backward_acc_copies<16384>(N, real, per);
        default: return 0;
    }
}

cudaError_t run_forward(const AfParams& p, cudaStream_t st) { GRAF_DISPATCH_M(run_forward_m, p.M, p, st) }
cudaError_t run_spectral(const SpecParams& q, cudaStream_t st) { GRAF_DISPATCH_M(run_spectral_m, q.N, q, st) }
cudaError_t run_composite(const CompParams& q, int M, cudaStream_t st) { GRAF_DISPATCH_M(run_composite_m, M, q, st) }
cudaError_t run_loss(const AfParams& p, cudaStream_t st) {
    cudaError_t e;
    switch (p.M) {
        case 8: e = run_loss_m<8>(p, st); break;
        case 16: e = run_loss_m<16>(p, st); break;
        case 32: e = run_loss_m<32>(p, st); break;
        case 64: e = run_loss_m<64>(p, st); break;
        case 128: e = run_loss_m<128>(p, st); break;
        case 256: e = run_loss_m<256>(p, st); break;
        case 512: e = run_loss_m<512>(p, st); break;
        case 1024: e = run_loss_m<1024>(p, st); break;
        case 2048: e = run_loss_m<2048>(p, st); break;
        case 4096: e = run_loss_m<4096>(p, st); break;
        case 8192: e = run_loss_m<8192>(p, st); break;
        case 16384: e = run_loss_m<16384>(p, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return run_finalize(p, st);
}
cudaError_t run_grad_reduce(const AfParams& p, const float* dL, float2* grad_s, float* grad_phi,
                            cudaStream_t st) {
    cudaError_t e;
    const long long grid = (long long)((p.N + 255) / 256) * p.B;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (!grad_s) {
        grad_phi_kernel<<<(unsigned)grid, 256, 0, st>>>(p, dL, grad_phi);
        return cudaGetLastError();
    }
    const size_t sm = (size_t)p.N * sizeof(double);
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute(uniform_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(grad_s_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    uniform_sum_kernel<<<p.B, 256, sm, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    grad_s_kernel<<<(unsigned)grid, 256, sm, st>>>(p, dL, grad_s, grad_phi);
    return cudaGetLastError();
}

cudaError_t run_backward_rows(const AfParams& p, cudaStream_t st) { GRAF_DISPATCH_M(run_backward_m, p.M, p, st) }
cudaError_t run_loss_rows(const AfParams& p, cudaStream_t st) { GRAF_DISPATCH_M(run_loss_m, p.M, p, st) }

cudaError_t run_backward(const AfParams& p, const float* dL, float2* grad_s, float* grad_phi,
                         cudaStream_t st) {
    cudaError_t e;
    switch (p.M) {
        case 8: e = run_backward_m<8>(p, st); break;
        case 16: e = run_backward_m<16>(p, st); break;
        case 32: e = run_backward_m<32>(p, st); break;
        case 64: e = run_backward_m<64>(p, st); break;
        case 128: e = run_backward_m<128>(p, st); break;
        case 256: e = run_backward_m<256>(p, st); break;
        case 512: e = run_backward_m<512>(p, st); break;
        case 1024: e = run_backward_m<1024>(p, st); break;
        case 2048: e = run_backward_m<2048>(p, st); break;
        case 4096: e = run_backward_m<4096>(p, st); break;
        case 8192: e = run_backward_m<8192>(p, st); break;
        case 16384: e = run_backward_m<16384>(p, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || !(grad_s || grad_phi)) return e;
    return run_grad_reduce(p, dL, grad_s, grad_phi, st);
}

cudaError_t run_fused(const AfParams& p, cudaStream_t st) { GRAF_DISPATCH_M(run_fused_m, p.M, p, st) }

static cudaError_t run_match_rows(const AfParams& p, cudaStream_t st) { GRAF_DISPATCH_M(run_match_m, p.M, p, st) }

cudaError_t run_match(const AfParams& p, float* loss_out, cudaStream_t st) {
    cudaError_t e = run_match_rows(p, st);
    if (e != cudaSuccess) return e;
    match_finalize_kernel<<<(p.B + 127) / 128, 128, 0, st>>>(p, loss_out);
    return cudaGetLastError();
}

cudaError_t run_peak_grad(const AfParams& p, const float* dL, float2* grad_s, float* grad_phi, int accumulate,
                          cudaStream_t st) {
    const size_t sm = (size_t)p.N * sizeof(float2);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(peak_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    peak_grad_kernel<<<p.B, 256, sm, st>>>(p, dL, grad_s, grad_phi, accumulate);
    return cudaGetLastError();
}

cudaError_t run_finalize(const AfParams& p, cudaStream_t st) {
    const int wpb = 4;
    loss_finalize_kernel<<<(p.B + wpb - 1) / wpb, 32 * wpb, 0, st>>>(p, p.out8);
    return cudaGetLastError();
}

}  // namespace graf

extern "C" {

graf_status_t graf_get_device_error_word(uint32_t* word, void* stream) {
    if (!word) return GRAF_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int h = 0;
    graf::take_device_error_kernel<<<1, 1, 0, st>>>();
    if (cudaGetLastError() != cudaSuccess) return GRAF_ERR_CUDA;
    if (cudaMemcpyFromSymbolAsync(&h, graf::g_device_error_taken, sizeof h, 0, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return GRAF_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GRAF_ERR_CUDA;
    *word = h;
    return GRAF_OK;
}

graf_status_t graf_get_device_error(void* stream) {
    uint32_t w = 0;
    const graf_status_t s = graf_get_device_error_word(&w, stream);
    if (s != GRAF_OK) return s;
    return w ? GRAF_ERR_DEVICE_FLAG : GRAF_OK;
}

}  // extern "C"
