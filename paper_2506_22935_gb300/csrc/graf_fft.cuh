// graf_fft.cuh - row DFTs of the ambiguity function, in registers and shared
// memory, for one GB300 SM.
//
// Computes X[m] = sum_n x[n] exp(-2 pi j m n / M) (paper Eq. 11, the FFT over
// the time axis of each delay row) and its adjoint sum_m G[m] exp(+2 pi j m n
// / M) (the linear inverse-transform step of the backward pass, Sec. 4.2,
// unnormalised).
//
// Layout: a row of length M is owned by TPR = M / VALS threads, VALS = 32
// complex values per thread in registers (16 for M = 128 and 256, 64 for
// M = 64, M below; see RowPlan).  On entry AND on exit thread t
// holds element t + TPR * w in register w ("natural strided" layout), so the
// lag-product builder, the loss epilogue and the gradient scatter all index
// the same way and the forward and inverse transforms chain without any
// reordering.
//
// Algorithm: Stockham auto-sort passes (Cooley-Tukey with a self-sorting
// output index, as in Govindaraju et al., SC'08), radices R_0 = VALS, then
// M / VALS as one radix (M <= 1024) or 16 x (M / 512).  Pass p with radix R and span Ns
// takes, for butterfly j, inputs x[j + r M/R], multiplies input r by
// W_(Ns R)^((j mod Ns) r), does an R-point DFT in registers and writes
// output r to (j / Ns) Ns R + (j mod Ns) + r Ns.  The first pass reads
// registers, the last keeps its outputs in registers; only the exchanges
// between passes go through shared memory (one for M <= 1024, two above).  Each
// R-point DFT is itself split A x B (A in {2,4,8}) with compile-time
// twiddles, so W_R^q folds into immediates.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "twiddles.inc"

namespace graf {

// ----------------------------------------------------------------- complex ops
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by -j (forward) or +j (inverse)
template <bool INV>
__host__ __device__ __forceinline__ float2 rot_mj(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int I, int N, class F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        sfor<I + 1, N>(f);
    }
}

// a * W_R^Q (forward) or a * conj(W_R^Q) (inverse), Q compile-time, R | 64
template <int R, int Q, bool INV>
__host__ __device__ __forceinline__ float2 twc(float2 a) {
    constexpr int q64 = (((Q % R) + R) % R) * (64 / R);
    if constexpr (q64 == 0) {
        return a;
    } else if constexpr (q64 == 16) {
        return rot_mj<INV>(a);
    } else if constexpr (q64 == 32) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (q64 == 48) {
        return rot_mj<!INV>(a);
    } else if constexpr ((q64 & 15) == 8) {
        // |Re W| = |Im W| = sqrt(1/2): two adds and two multiplies
        constexpr float c = graf_w64_re(q64);
        constexpr float s = INV ? -graf_w64_im(q64) : graf_w64_im(q64);
        constexpr float h = c > 0.0f ? c : -c;
        constexpr float sc = c > 0.0f ? 1.0f : -1.0f;
        constexpr float ss = s > 0.0f ? 1.0f : -1.0f;
        return make_float2(h * (sc * a.x - ss * a.y), h * (ss * a.x + sc * a.y));
    } else {
        constexpr float c = graf_w64_re(q64);
        constexpr float s = INV ? -graf_w64_im(q64) : graf_w64_im(q64);
        return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
    }
}

// ---------------------------------------------------- in-register DFT kernels
// dft<R, OFF, ST, INV, HIN, HOUT>(v): in-place R-point DFT of the values
// v[OFF + ST*i], i in [0,R), output X[k] at v[OFF + ST*k].
//   HIN : inputs i >= R/2 are known zero (zero-padded row, N <= M/2)
//   HOUT: only outputs k < R/2 are needed (the rest is left unspecified)

template <int OFF, int ST, bool INV, bool HIN, bool HOUT>
__host__ __device__ __forceinline__ void dft2(float2* v) {
    float2 a = v[OFF], b = v[OFF + ST];
    if constexpr (HIN) {
        v[OFF + ST] = a;
    } else {
        v[OFF] = cadd(a, b);
        if constexpr (!HOUT) v[OFF + ST] = csub(a, b);
    }
}

template <int OFF, int ST, bool INV, bool HIN, bool HOUT>
__host__ __device__ __forceinline__ void dft4(float2* v) {
    float2 a0 = v[OFF], a1 = v[OFF + ST], a2 = v[OFF + 2 * ST], a3 = v[OFF + 3 * ST];
    float2 s02, d02, s13, d13;
    if constexpr (HIN) {
        s02 = a0; d02 = a0; s13 = a1; d13 = rot_mj<INV>(a1);
    } else {
        s02 = cadd(a0, a2); d02 = csub(a0, a2);
        s13 = cadd(a1, a3); d13 = rot_mj<INV>(csub(a1, a3));
    }
    v[OFF] = cadd(s02, s13);
    v[OFF + ST] = cadd(d02, d13);
    if constexpr (!HOUT) {
        v[OFF + 2 * ST] = csub(s02, s13);
        v[OFF + 3 * ST] = csub(d02, d13);
    }
}

template <int OFF, int ST, bool INV, bool HIN, bool HOUT>
__host__ __device__ __forceinline__ void dft8(float2* v) {
    // radix-2 split: even/odd samples, X[q] = E[q] + W8^q O[q], X[q+4] = E[q] - W8^q O[q]
    dft4<OFF, 2 * ST, INV, HIN, false>(v);
    dft4<OFF + ST, 2 * ST, INV, HIN, false>(v);
    float2 e[4], o[4];
    sfor<0, 4>([&](auto q) {
        e[q] = v[OFF + 2 * ST * q];
        o[q] = twc<8, decltype(q)::value, INV>(v[OFF + ST + 2 * ST * q]);
    });
    sfor<0, 4>([&](auto q) {
        v[OFF + ST * q] = cadd(e[q], o[q]);
        if constexpr (!HOUT) v[OFF + ST * (q + 4)] = csub(e[q], o[q]);
    });
}

template <int R, int OFF, int ST, bool INV, bool HIN, bool HOUT>
__host__ __device__ __forceinline__ void dft(float2* v);

// R = A * B four-step in registers: n = b + B a, k = d + A c.
//   1. for each b: A-point DFT over a of v[b + B a]      -> Y_b[d] at slot b + B d
//   2. Y_b[d] *= W_R^(b d)
//   3. for each d: B-point DFT over b of Y_b[d]          -> X[d + A c] at slot B d + c
//   4. permute registers to natural order (renaming only)
template <int R, int A, int OFF, int ST, bool INV, bool HIN, bool HOUT>
__host__ __device__ __forceinline__ void dft_split(float2* v) {
    constexpr int B = R / A;
    sfor<0, B>([&](auto b) { dft<A, OFF + ST * decltype(b)::value, ST * B, INV, HIN, false>(v); });
    sfor<1, B>([&](auto b) {
        sfor<1, A>([&](auto d) {
            constexpr int bi = decltype(b)::value, di = decltype(d)::value;
            v[OFF + ST * (bi + B * di)] = twc<R, bi * di, INV>(v[OFF + ST * (bi + B * di)]);
        });
    });
    sfor<0, A>([&](auto d) { dft<B, OFF + ST * B * decltype(d)::value, ST, INV, false, HOUT>(v); });
    float2 t[R];
    sfor<0, A>([&](auto d) {
        sfor<0, B>([&](auto c) {
            constexpr int di = decltype(d)::value, ci = decltype(c)::value;
            t[di + A * ci] = v[OFF + ST * (B * di + ci)];
        });
    });
    sfor<0, R>([&](auto k) { v[OFF + ST * decltype(k)::value] = t[k]; });
}

template <int R, int OFF, int ST, bool INV, bool HIN, bool HOUT>
__host__ __device__ __forceinline__ void dft(float2* v) {
    static_assert(R == 1 || R == 2 || R == 4 || R == 8 || R == 16 || R == 32 || R == 64,
                  "radix must be a power of two up to 64");
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2<OFF, ST, INV, HIN, HOUT>(v);
    } else if constexpr (R == 4) {
        dft4<OFF, ST, INV, HIN, HOUT>(v);
    } else if constexpr (R == 8) {
        dft8<OFF, ST, INV, HIN, HOUT>(v);
    } else if constexpr (R == 16) {
        dft_split<16, 4, OFF, ST, INV, HIN, HOUT>(v);
    } else {
        dft_split<R, 8, OFF, ST, INV, HIN, HOUT>(v);
    }
}

// ------------------------------------------------------------------ row plan
// V = 1 (M = 8192 only): two row slots per CTA of 512 threads, each with a
// whole exchange buffer (no real/imaginary split) -- the plan of the fused
// kernel when the signal is short enough for both buffers to fit (N <= M/2,
// phase gradient only).
template <int M, int V = 0>
struct RowPlan {
    static_assert(M >= 8 && M <= 16384 && (M & (M - 1)) == 0, "M must be a power of two in [8,16384]");
    // values per thread: 32 from M = 512 on, so that a thread needs at most
    // 128 registers and 16 warps share an SM (two CTAs of 256 threads, or one
    // of 512 threads for M = 16384, whose row spans 512 threads); a third FFT
    // pass from M = 2048 on is the price.  16 for M = 128 and 256 (still two
    // passes; the fused kernel's per-row state then fits 128 registers
    // without spilling).  64 for M = 64, M below.
    static constexpr int VALS = M >= 512 ? 32 : (M >= 128 ? 16 : (M < 64 ? M : 64));
    static constexpr int TPR = M / VALS;           // threads per row
    static_assert(V == 0 || M == 8192, "the two-slot plan exists for M = 8192 only");
    static constexpr int THREADS = V == 1 ? 2 * TPR : (TPR > 256 ? TPR : 256);  // threads per CTA
    static constexpr int NPASS = TPR == 1 ? 1 : (TPR <= VALS ? 2 : 3);
    static constexpr int R0 = VALS;
    static constexpr int R1 = NPASS == 1 ? 1 : (NPASS == 2 ? TPR : 16);
    static constexpr int R2 = NPASS == 3 ? TPR / 16 : 1;
    static constexpr int MIN_BLOCKS = ((VALS == 32 || VALS == 16) && THREADS == 256) ? 2 : 1;  // CTAs per SM the registers allow
    // shared-memory row buffer (float2 units): one pad slot per VALS values
    // keeps the stride-VALS stores of the first pass free of bank conflicts
    static constexpr int PAD = VALS < 16 ? 64 : VALS;
    static constexpr int SMEM_ROW = NPASS == 1 ? 0 : M + M / PAD;
    // exchange real and imaginary halves separately (half the buffer) for the
    // largest rows so that the backward's accumulators still fit
    static constexpr bool SPLIT = V == 0 && M >= 8192;
};

template <int PAD>
__device__ __forceinline__ int padi(int i) { return i + i / PAD; }

template <int M, int P>
__device__ __forceinline__ const float2* tw_table() {
    return GrafTw<M, P>::get();
}

// Barrier over the TPR threads of one row (a warp or less: __syncwarp; more:
// a named barrier per row slot, ids 1..15; id 0 stays __syncthreads').
template <int TPR>
__device__ __forceinline__ void row_sync(int slot) {
    if constexpr (TPR <= 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(slot + 1), "r"(TPR) : "memory");
    }
}

// Shared-memory addressing.  Logical element i of a row lives at padi(i) =
// i + i/64.  Every access below is written as a per-thread base pointer plus
// a compile-time offset, so no per-element address stays live in registers.
//
// Store of pass p (radix R, span NS): butterfly j = t + TPR u writes output r
// to element (j / NS) NS R + (j mod NS) + r NS.  For NS = 1 this is j R + r
// (padded: 65 j + r, R = 64); for NS a multiple of 64 the padded address is
// padi(idxD) + 65 r (NS/64).
template <int M, int R, int NS, bool SPLIT_PART_RE, bool SPLIT>
__device__ __forceinline__ void pass_store(const float2* v, float2* buf, int t) {
    using P = RowPlan<M>;
    constexpr int NB = P::VALS / R;
    constexpr int PAD = P::PAD;
    static_assert(NS == 1 || NS % PAD == 0, "pass span must be 1 or a multiple of the pad period");
    static_assert(NS != 1 || (R == PAD && NB == 1), "first pass must be radix VALS");
    sfor<0, NB>([&](auto u) {
        const int j = t + P::TPR * decltype(u)::value;
        int base;
        if constexpr (NS == 1) {
            base = (PAD + 1) * j;
        } else {
            base = padi<PAD>((j / NS) * NS * R + (j % NS));
        }
        sfor<0, R>([&](auto r) {
            constexpr int off = NS == 1 ? decltype(r)::value : decltype(r)::value * (NS + NS / PAD);
            const float2 x = v[decltype(u)::value * R + decltype(r)::value];
            if constexpr (!SPLIT) buf[base + off] = x;
            else reinterpret_cast<float*>(buf)[base + off] = SPLIT_PART_RE ? x.x : x.y;
        });
    });
}

// Load of pass p (radix R): butterfly j = t + TPR u reads element j + r M/R
// into v[u R + r]; M/R is a multiple of 64 and j < M/R, so the padded address
// is padi(j) + r (M/R)(65/64).
template <int M, int R, bool SPLIT_PART_RE, bool SPLIT>
__device__ __forceinline__ void pass_load(float2* v, const float2* buf, int t) {
    using P = RowPlan<M>;
    constexpr int NB = P::VALS / R;
    constexpr int STRIDE = M / R;
    static_assert(STRIDE % P::PAD == 0, "load stride must be a multiple of the pad period");
    sfor<0, NB>([&](auto u) {
        const int j = t + P::TPR * decltype(u)::value;
        const int base = padi<P::PAD>(j);
        sfor<0, R>([&](auto r) {
            constexpr int off = decltype(r)::value * (STRIDE + STRIDE / P::PAD);
            float2& x = v[decltype(u)::value * R + decltype(r)::value];
            if constexpr (!SPLIT) x = buf[base + off];
            else if constexpr (SPLIT_PART_RE) x.x = reinterpret_cast<const float*>(buf)[base + off];
            else x.y = reinterpret_cast<const float*>(buf)[base + off];
        });
    });
}

// Exchange through shared memory between pass p (radix RS, span NSS) and
// pass p+1 (radix RL): store, barrier, load.  The caller guarantees the buffer
// is free on entry (a barrier since its last reads).
template <int M, int RS, int NSS, int RL, int V = 0>
__device__ __forceinline__ void exchange(float2* v, float2* buf, int t, int slot) {
    using P = RowPlan<M, V>;
    if constexpr (!P::SPLIT) {
        pass_store<M, RS, NSS, true, false>(v, buf, t);
        row_sync<P::TPR>(slot);
        pass_load<M, RL, true, false>(v, buf, t);
    } else {
        // half-size buffer: real parts first, then imaginary parts
        float lre[P::VALS];
        pass_store<M, RS, NSS, true, true>(v, buf, t);
        row_sync<P::TPR>(slot);
        {
            constexpr int NB = P::VALS / RL;
            constexpr int STRIDE = M / RL;
            sfor<0, NB>([&](auto u) {
                const int base = padi<P::PAD>(t + P::TPR * decltype(u)::value);
                sfor<0, RL>([&](auto r) {
                    constexpr int off = decltype(r)::value * (STRIDE + STRIDE / P::PAD);
                    lre[decltype(u)::value * RL + decltype(r)::value] = reinterpret_cast<const float*>(buf)[base + off];
                });
            });
        }
        row_sync<P::TPR>(slot);
        pass_store<M, RS, NSS, false, true>(v, buf, t);
        row_sync<P::TPR>(slot);
        pass_load<M, RL, false, true>(v, buf, t);
        sfor<0, P::VALS>([&](auto i) { v[i].x = lre[i]; });
    }
}

// Read-only twiddle load.  The volatile asm keeps the compiler from hoisting
// the (row-invariant) loads out of the row loop, which would pin up to 124
// registers per thread for the whole kernel.
__device__ __forceinline__ float2 ld_tw(const float2* p) {
    float2 r;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
    return r;
}

// Twiddle and DFT of pass p >= 1 (radix R, span NS): input r of butterfly j
// is multiplied by W_(NS R)^((j mod NS) r), read from the pass's table at
// [(r-1) NS + (j mod NS)] (base pointer + immediate offset).
template <int M, int P_, int R, int NS, bool INV, bool HOUT>
__device__ __forceinline__ void pass_compute(float2* v, int t) {
    using P = RowPlan<M>;
    constexpr int NB = P::VALS / R;
    if constexpr (NB > 1 && P::TPR % NS == 0) {
        // j mod NS = t mod NS for every butterfly j = t + TPR u of this
        // thread: one load of each twiddle serves all of them
        const float2* tw = tw_table<M, P_>() + (t % NS);
        sfor<1, R>([&](auto r) {
            const float2 w = ld_tw(tw + (decltype(r)::value - 1) * NS);
            sfor<0, NB>([&](auto u) {
                float2& x = v[decltype(u)::value * R + decltype(r)::value];
                x = INV ? cmulc(x, w) : cmul(x, w);
            });
        });
        sfor<0, NB>([&](auto u) { dft<R, decltype(u)::value * R, 1, INV, false, HOUT>(v); });
        return;
    }
    sfor<0, NB>([&](auto u) {
        const int j = t + P::TPR * decltype(u)::value;
        const float2* tw = tw_table<M, P_>() + (j % NS);
        sfor<1, R>([&](auto r) {
            const float2 w = ld_tw(tw + (decltype(r)::value - 1) * NS);
            float2& x = v[decltype(u)::value * R + decltype(r)::value];
            x = INV ? cmulc(x, w) : cmul(x, w);
        });
        dft<R, decltype(u)::value * R, 1, INV, false, HOUT>(v);
    });
}

// Register permutation after the last pass (radix R): output r of butterfly
// u sits at v[u R + r] and is element t + TPR (u + NB r) of the row.
template <int VALS, int R>
__device__ __forceinline__ void final_permute(float2* v) {
    constexpr int NB = VALS / R;
    if constexpr (NB > 1) {
        float2 tmp[VALS];
        sfor<0, NB>([&](auto u) {
            sfor<0, R>([&](auto r) {
                tmp[decltype(u)::value + NB * decltype(r)::value] = v[decltype(u)::value * R + decltype(r)::value];
            });
        });
        sfor<0, VALS>([&](auto i) { v[i] = tmp[i]; });
    }
}

// Full row transform, natural strided layout in and out.
//   INV : adjoint (conjugate twiddles, no 1/M scaling)
//   HIN : inputs with n >= M/2 are zero (the lag row of a waveform with N <= M/2)
//   HOUT: only outputs n < M/2 are needed
// `buf` is this row's shared-memory buffer (RowPlan<M>::SMEM_ROW float2),
// free on entry; on exit it may still be read by other threads of the row
// until the next row_sync.
template <int M, bool INV, bool HIN, bool HOUT, int V = 0>
__device__ __forceinline__ void row_fft(float2* v, float2* buf, int t, int slot) {
    using P = RowPlan<M, V>;
    if constexpr (P::NPASS == 1) {
        dft<P::R0, 0, 1, INV, HIN, HOUT>(v);
    } else if constexpr (P::NPASS == 2) {
        dft<P::R0, 0, 1, INV, HIN, false>(v);
        exchange<M, P::R0, 1, P::R1, V>(v, buf, t, slot);
        pass_compute<M, 1, P::R1, P::R0, INV, HOUT>(v, t);
        final_permute<P::VALS, P::R1>(v);
    } else {
        dft<P::R0, 0, 1, INV, HIN, false>(v);
        exchange<M, P::R0, 1, P::R1, V>(v, buf, t, slot);
        pass_compute<M, 1, P::R1, P::R0, INV, false>(v, t);
        row_sync<P::TPR>(slot);
        exchange<M, P::R1, P::R0, P::R2, V>(v, buf, t, slot);
        pass_compute<M, 2, P::R2, P::R0 * P::R1, INV, HOUT>(v, t);
        final_permute<P::VALS, P::R2>(v);
    }
}

}  // namespace graf
