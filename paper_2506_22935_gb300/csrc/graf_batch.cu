// graf_batch.cu - batches of waveforms of unequal length (each with its own
// Doppler length, window and loss weights) in persistent launches, one per
// row length M, fed from a longest-first work list, with an autotuned tile
// size per M.  The paper's batch processing (Sec. 4.3: s in C^{B x N}) made
// ragged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "graf.h"
#include "graf_kernels.cuh"

using graf::AfParams;
using graf::WaveDesc;

namespace {

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Bucket {
    int M = 0;
    int rps = 0;          // rows per slot and tile (tile = slots x rps rows)
    bool fused = true;    // fused loss + gradient, else loss then recomputing backward
    int acc_copies = 0;
    int max_N = 0;
    std::vector<int> waves;       // waveforms in this bucket
    std::vector<int2> items;      // (waveform, tile), longest first
    int2* d_items = nullptr;
    int item_begin = 0;           // first record index of the bucket's items
};

}  // namespace

struct graf_batch_plan_s {
    int B = 0;
    graf_input_t kind = GRAF_IN_PHASE;
    std::vector<WaveDesc> waves;
    std::vector<Bucket> buckets;
    WaveDesc* d_waves = nullptr;
    unsigned int* d_counters = nullptr;
    long long total_x = 0;     // sum of N
    int total_items = 0;
    long long total_gpart = 0; // float2 count of all gradient partials
    int max_N = 0;
    size_t ws_rec = 0, ws_scale = 0, ws_csum = 0, ws_gpart = 0, ws_usum = 0;
    // multi-scenario plans (Eq. 24): entry b scores source waveform src[b];
    // entry gradients go to a scratch area and are summed per source
    bool scenarios = false;
    int B_src = 0;
    std::vector<int> src;
    std::vector<long long> src_off;   // [B_src + 1] packed offsets of the sources
    int* d_src_entries = nullptr;     // entries grouped by source, ascending
    int* d_src_first = nullptr;       // [B_src + 1] CSR into d_src_entries
    long long* d_src_off = nullptr;   // [B_src + 1]
    size_t ws_scratch = 0;            // float (phase) or float2 (complex) per entry sample
    long long total_af = 0;           // floats of the packed forward output
    std::vector<long long> af_off;    // [B + 1] offsets of the waveforms' windows in it
};

namespace {

// Lay out tiles, work items and workspace for the current per-bucket rps.
graf_status_t layout(graf_batch_plan_s* P) {
    P->total_items = 0;
    P->total_gpart = 0;
    for (Bucket& bk : P->buckets) {
        const int slots = graf::slots_of(bk.M);
        const int rpt = slots * bk.rps;
        bk.items.clear();
        std::vector<std::pair<long long, int2>> cost;
        for (int b : bk.waves) {
            WaveDesc& d = P->waves[b];
            d.rows_per_tile = rpt;
            d.tiles = (d.r_hi - d.r_lo + 1 + rpt - 1) / rpt;
            for (int tl = 0; tl < d.tiles; ++tl) {
                const int rows = std::min(rpt, d.r_hi - (d.r_lo + tl * rpt) + 1);
                // rows x (M log M transform + N-long lag product and scatter)
                const long long c = (long long)rows * ((long long)bk.M * 11 + 4LL * d.N);
                cost.push_back({c, make_int2(b, tl)});
            }
        }
        std::stable_sort(cost.begin(), cost.end(),
                         [](const std::pair<long long, int2>& a, const std::pair<long long, int2>& c) {
                             return a.first > c.first;
                         });
        for (auto& c : cost) bk.items.push_back(c.second);
    }
    // per-waveform record and partial offsets (items of one waveform contiguous)
    int rec = 0;
    long long gp = 0;
    for (int b = 0; b < P->B; ++b) {
        WaveDesc& d = P->waves[b];
        d.rec_off = rec;
        d.gpart_off = gp;
        rec += d.tiles;
        gp += (long long)d.tiles * d.N;
    }
    P->total_items = rec;
    P->total_gpart = gp;
    P->ws_rec = align256((size_t)rec * sizeof(float4));
    P->ws_scale = align256((size_t)rec * sizeof(float));
    P->ws_csum = align256((size_t)rec * sizeof(float));
    P->ws_gpart = align256((size_t)gp * sizeof(float2));
    P->ws_usum = align256((size_t)2 * P->B * sizeof(double));
    P->ws_scratch = P->scenarios ? align256((size_t)P->total_x * (P->kind == GRAF_IN_PHASE ? sizeof(float)
                                                                                           : sizeof(float2)))
                                 : 0;
    // device copies
    cudaError_t e = cudaMemcpy(P->d_waves, P->waves.data(), sizeof(WaveDesc) * P->B, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return GRAF_ERR_CUDA;
    for (Bucket& bk : P->buckets) {
        if (bk.d_items) cudaFree(bk.d_items);
        bk.d_items = nullptr;
        if (cudaMalloc(&bk.d_items, sizeof(int2) * bk.items.size()) != cudaSuccess) return GRAF_ERR_NOMEM;
        if (cudaMemcpy(bk.d_items, bk.items.data(), sizeof(int2) * bk.items.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return GRAF_ERR_CUDA;
    }
    return GRAF_OK;
}

AfParams bucket_params(const graf_batch_plan_s* P, const Bucket& bk, int bi, const void* x, void* ws,
                       float* out8) {
    AfParams p{};
    p.x = x;
    p.kind = P->kind == GRAF_IN_PHASE ? 1 : 0;
    p.B = P->B;
    p.N = bk.max_N;
    p.M = bk.M;
    p.waves = P->d_waves;
    p.items = bk.d_items;
    p.n_items = (int)bk.items.size();
    p.counter = P->d_counters + bi;
    if (ws) {  // (the forward call has no workspace)
        unsigned char* w = static_cast<unsigned char*>(ws);
        p.rec = reinterpret_cast<float4*>(w);
        p.scale = reinterpret_cast<float*>(w + P->ws_rec);
        p.csum = reinterpret_cast<float*>(w + P->ws_rec + P->ws_scale);
        p.gpart = reinterpret_cast<float2*>(w + P->ws_rec + P->ws_scale + P->ws_csum);
        p.usum = reinterpret_cast<double*>(w + P->ws_rec + P->ws_scale + P->ws_csum + P->ws_gpart);
    }
    p.out8 = out8;
    p.saved8 = out8;
    p.phase_only = P->kind == GRAF_IN_PHASE ? 1 : 0;
    p.acc_copies = bk.acc_copies;
    p.defer_hi = -1;
    return p;
}

graf_status_t run_rows(const graf_batch_plan_s* P, const Bucket& bk, int bi, const void* x, void* ws,
                       float* out8, int which, cudaStream_t st) {
    AfParams p = bucket_params(P, bk, bi, x, ws, out8);
    if (cudaMemsetAsync(p.counter, 0, sizeof(unsigned int), st) != cudaSuccess) return GRAF_ERR_CUDA;
    cudaError_t e = which == 0 ? graf::run_fused(p, st)
                  : which == 1 ? graf::run_loss_rows(p, st)
                               : graf::run_backward_rows(p, st);
    return e == cudaSuccess ? GRAF_OK : GRAF_ERR_CUDA;
}

// Multi-scenario sum (Eq. 24): grad[j][n] = sum over the entries b of source
// j, in ascending order, of the entry gradient at waves[b].out_off + n (each
// already scaled by its weight dL[b] = lambda_b).  One thread per float of
// the gradient: `width` floats per sample (1 phase, 2 complex).
__global__ void scenario_sum_kernel(const WaveDesc* waves, const int* entries, const int* first,
                                    const long long* src_off, int B_src, int width, const float* scratch,
                                    float* grad) {
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= src_off[B_src] * width) return;
    const long long i = f / width;
    const int c = (int)(f - i * width);
    int lo = 0, hi = B_src - 1;  // source j with src_off[j] <= i < src_off[j+1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (src_off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const long long n = i - src_off[lo];
    float s = 0.0f;
    for (int e = first[lo]; e < first[lo + 1]; ++e) s += scratch[(waves[entries[e]].out_off + n) * width + c];
    grad[f] = s;
}

// The loss rows of every bucket (loss kernel or fused kernel), then the
// finalisation.
graf_status_t batch_loss_rows(const graf_batch_plan_s* P, const void* x, float* out8, void* ws, bool fused_ok,
                              bool* any_two_pass, cudaStream_t st) {
    graf_status_t s;
    *any_two_pass = false;
    for (size_t i = 0; i < P->buckets.size(); ++i) {
        const Bucket& bk = P->buckets[i];
        if (bk.fused && fused_ok) s = run_rows(P, bk, (int)i, x, ws, out8, 0, st);
        else {
            *any_two_pass = *any_two_pass || fused_ok;
            s = run_rows(P, bk, (int)i, x, ws, out8, 1, st);
        }
        if (s != GRAF_OK) return s;
    }
    AfParams q = bucket_params(P, P->buckets[0], 0, x, ws, out8);
    q.N = P->max_N;
    if (graf::run_finalize(q, st) != cudaSuccess) return GRAF_ERR_CUDA;
    return GRAF_OK;
}

// The whole step for all buckets on one stream: loss scalars, then the
// gradient (grad_phi for phase plans, grad_s for complex ones).
graf_status_t batch_step(const graf_batch_plan_s* P, const void* x, float* out8, const float* dL, float2* grad_s,
                         float* grad_phi, void* ws, cudaStream_t st) {
    bool any_two_pass = false;
    graf_status_t s = batch_loss_rows(P, x, out8, ws, true, &any_two_pass, st);
    if (s != GRAF_OK) return s;
    if (any_two_pass)
        for (size_t i = 0; i < P->buckets.size(); ++i)
            if (!P->buckets[i].fused && (s = run_rows(P, P->buckets[i], (int)i, x, ws, out8, 2, st)) != GRAF_OK)
                return s;
    AfParams q = bucket_params(P, P->buckets[0], 0, x, ws, out8);
    q.N = P->max_N;
    if (!P->scenarios) {
        if (graf::run_grad_reduce(q, dL, grad_s, grad_phi, st) != cudaSuccess) return GRAF_ERR_CUDA;
        return GRAF_OK;
    }
    float* scratch = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) + P->ws_rec + P->ws_scale +
                                              P->ws_csum + P->ws_gpart + P->ws_usum);
    const int width = grad_s ? 2 : 1;
    if (graf::run_grad_reduce(q, dL, grad_s ? reinterpret_cast<float2*>(scratch) : nullptr,
                              grad_s ? nullptr : scratch, st) != cudaSuccess)
        return GRAF_ERR_CUDA;
    const long long n_src = P->src_off[P->B_src] * width;
    const unsigned grid = (unsigned)((n_src + 255) / 256);
    scenario_sum_kernel<<<grid, 256, 0, st>>>(P->d_waves, P->d_src_entries, P->d_src_first, P->d_src_off,
                                              P->B_src, width, scratch,
                                              grad_s ? reinterpret_cast<float*>(grad_s) : grad_phi);
    return cudaGetLastError() == cudaSuccess ? GRAF_OK : GRAF_ERR_CUDA;
}

graf_status_t validate_window(int N, int M, const graf_window_t& w) {
    if (w.k_lo > w.k_hi || w.m_lo > w.m_hi) return GRAF_ERR_INVALID_ARG;
    if (w.k_lo < -(N - 1) || w.k_hi > N - 1) return GRAF_ERR_INVALID_ARG;
    if (w.m_lo < -(M / 2) || w.m_hi > M / 2 - 1) return GRAF_ERR_INVALID_ARG;
    if (w.k_ml < -1 || w.m_ml < -1) return GRAF_ERR_INVALID_ARG;
    return GRAF_OK;
}

}  // namespace

extern "C" {

// Plan entries b = 0..B-1.  Plain plans: entry b is waveform b of length
// N_host[b].  Multi-scenario plans (src_host set): entry b scores source
// waveform src_host[b] (length N_src_host[src]) with its own M, window and loss.
static graf_status_t create_plan(int32_t B, const int32_t* N_host, const int32_t* M_host,
                                 const graf_window_t* w_host, const graf_loss_t* l_host,
                                 int32_t losses_per_waveform, graf_input_t kind, const int32_t* src_host,
                                 int32_t B_src, const int32_t* N_src_host, graf_batch_plan_t* plan) {
    if (!plan) return GRAF_ERR_INVALID_ARG;
    *plan = nullptr;
    if (B < 1 || B > (1 << 20) || !l_host) return GRAF_ERR_INVALID_ARG;
    if (src_host ? (!N_src_host || B_src < 1 || B_src > (1 << 20)) : !N_host) return GRAF_ERR_INVALID_ARG;
    if (kind != GRAF_IN_PHASE && kind != GRAF_IN_COMPLEX) return GRAF_ERR_INVALID_ARG;
    graf_batch_plan_s* P = new (std::nothrow) graf_batch_plan_s();
    if (!P) return GRAF_ERR_NOMEM;
    P->B = B;
    P->kind = kind;
    P->waves.resize(B);
    if (src_host) {
        P->scenarios = true;
        P->B_src = B_src;
        P->src.assign(src_host, src_host + B);
        P->src_off.assign((size_t)B_src + 1, 0);
        for (int j = 0; j < B_src; ++j) {
            if (N_src_host[j] < 1) {
                delete P;
                return GRAF_ERR_INVALID_ARG;
            }
            P->src_off[j + 1] = P->src_off[j] + N_src_host[j];
        }
        for (int b = 0; b < B; ++b)
            if (src_host[b] < 0 || src_host[b] >= B_src) {
                delete P;
                return GRAF_ERR_INVALID_ARG;
            }
    }
    long long off = 0;
    std::vector<int> Ms;
    for (int b = 0; b < B; ++b) {
        const int N = src_host ? N_src_host[src_host[b]] : N_host[b];
        const int M = M_host ? M_host[b] : next_pow2(2 * N);
        const graf_loss_t& l = l_host[losses_per_waveform ? b : 0];
        if (N < 1 || M < GRAF_M_MIN || M > GRAF_M_MAX || (M & (M - 1)) || N > M || !(l.beta > 0.0f) ||
            !(l.eps >= 0.0f)) {
            delete P;
            return GRAF_ERR_INVALID_ARG;
        }
        if (graf::is_hard_beta(l.beta)) {  // the hard PSL runs through the single-shape calls only
            delete P;
            return GRAF_ERR_UNSUPPORTED;
        }
        graf_window_t w;
        if (w_host) w = w_host[b];
        else w = graf_window_t{-(N - 1), N - 1, -(M / 2), M / 2 - 1, 0, std::max(M / N - 1, 0)};
        if (validate_window(N, M, w) != GRAF_OK) {
            delete P;
            return GRAF_ERR_INVALID_ARG;
        }
        WaveDesc& d = P->waves[b];
        std::memset(&d, 0, sizeof(d));
        d.x_off = src_host ? P->src_off[src_host[b]] : off;
        d.out_off = off;  // scenario plans: the entry's gradient in the scratch area
        off += N;
        d.N = N;
        d.M = M;
        d.k_lo = w.k_lo; d.k_hi = w.k_hi; d.m_lo = w.m_lo; d.m_hi = w.m_hi; d.k_ml = w.k_ml; d.m_ml = w.m_ml;
        const graf::Tiling T = graf::make_tiling(1, M, w.k_lo, w.k_hi, 1);
        d.r_lo = T.r_lo;
        d.r_hi = T.r_hi;
        d.eps = l.eps; d.beta = l.beta; d.w_psl = l.w_psl; d.w_isl = l.w_isl;
        d.defer_hi = -1;
        d.af_off = P->total_af;
        P->af_off.push_back(P->total_af);
        P->total_af += (long long)(w.k_hi - w.k_lo + 1) * (w.m_hi - w.m_lo + 1);
        P->max_N = std::max(P->max_N, N);
        if (std::find(Ms.begin(), Ms.end(), M) == Ms.end()) Ms.push_back(M);
    }
    P->total_x = off;
    P->af_off.push_back(P->total_af);
    std::sort(Ms.begin(), Ms.end(), [](int a, int c) { return a > c; });  // largest rows first
    for (int M : Ms) {
        std::vector<int> all;
        int max_N = 0;
        for (int b = 0; b < B; ++b)
            if (P->waves[b].M == M) {
                all.push_back(b);
                max_N = std::max(max_N, P->waves[b].N);
            }
        const int real = P->kind == GRAF_IN_PHASE ? 1 : 0;  // phase gradients use real accumulators
        const int acc = graf::acc_copies_for(M, max_N, real);
        if (acc < 1 || graf::row_kernel_smem(M, max_N, 0) > graf::kMaxSmem) {
            delete P;
            return GRAF_ERR_UNSUPPORTED;
        }
        // A waveform runs fused unless it has PSL over a window that does not
        // span every Doppler bin, or mainlobe-box rows beyond row 0 (row 0
        // carries no phase gradient), or its log-sum-exp shift is a running one
        // (it rescales the accumulators) and the slots cannot each own an
        // accumulator.  The fused and the two-pass waveforms of one M go to
        // separate buckets, so one of the latter does not slow the rest.
        const int slots = graf::slots_of(M);
        std::vector<int> fused, two_pass;
        for (int b : all) {
            WaveDesc& d = P->waves[b];
            const bool full_m = d.m_lo == -(M / 2) && d.m_hi == M / 2 - 1;
            const bool fixed = graf::lse_fixed_shift(P->kind == GRAF_IN_PHASE ? 1 : 0, d.eps, d.beta, d.N) > 0.0f;
            bool ok = true;
            if (d.w_psl != 0.0f) {
                if (!full_m || d.k_ml >= 1 || (!fixed && acc < slots)) ok = false;
                // a box on row 0: its cells' weights are not uniform, so the
                // fused kernel leaves row 0's gradient out; that is exact for
                // phase codes (row 0 does not depend on the phases), and a
                // complex waveform takes the two-pass path instead
                else if (d.k_ml == 0 && d.m_ml >= 0 && d.r_lo == 0) {
                    if (real) d.defer_hi = 0;
                    else ok = false;
                }
            }
            (ok ? fused : two_pass).push_back(b);
        }
        for (int pass = 0; pass < 2; ++pass) {
            const std::vector<int>& ws = pass == 0 ? fused : two_pass;
            if (ws.empty()) continue;
            Bucket bk;
            bk.M = M;
            bk.rps = 4;
            bk.fused = pass == 0;
            bk.waves = ws;
            for (int b : ws) bk.max_N = std::max(bk.max_N, P->waves[b].N);
            bk.acc_copies = graf::acc_copies_for(M, bk.max_N, real);
            for (int b : ws) {
                P->waves[b].unscaled = bk.fused ? 0 : 1;
                if (!bk.fused) P->waves[b].defer_hi = -1;
            }
            P->buckets.push_back(bk);
        }
    }
    if (cudaMalloc(&P->d_waves, sizeof(WaveDesc) * B) != cudaSuccess ||
        cudaMalloc(&P->d_counters, sizeof(unsigned int) * P->buckets.size()) != cudaSuccess) {
        graf_batch_plan_destroy(P);
        return GRAF_ERR_NOMEM;
    }
    graf_status_t s = layout(P);
    if (s != GRAF_OK) {
        graf_batch_plan_destroy(P);
        return s;
    }
    if (P->scenarios) {
        std::vector<int> first((size_t)B_src + 1, 0), entries;
        for (int j = 0; j < B_src; ++j) {
            first[j] = (int)entries.size();
            for (int b = 0; b < B; ++b)
                if (P->src[b] == j) entries.push_back(b);
        }
        first[B_src] = (int)entries.size();
        if (cudaMalloc(&P->d_src_entries, sizeof(int) * entries.size()) != cudaSuccess ||
            cudaMalloc(&P->d_src_first, sizeof(int) * first.size()) != cudaSuccess ||
            cudaMalloc(&P->d_src_off, sizeof(long long) * P->src_off.size()) != cudaSuccess) {
            graf_batch_plan_destroy(P);
            return GRAF_ERR_NOMEM;
        }
        if (cudaMemcpy(P->d_src_entries, entries.data(), sizeof(int) * entries.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(P->d_src_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(P->d_src_off, P->src_off.data(), sizeof(long long) * P->src_off.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            graf_batch_plan_destroy(P);
            return GRAF_ERR_CUDA;
        }
    }
    *plan = P;
    return GRAF_OK;
}

graf_status_t graf_batch_plan_create(int32_t B, const int32_t* N_host, const int32_t* M_host,
                                     const graf_window_t* w_host, const graf_loss_t* l_host,
                                     int32_t losses_per_waveform, graf_input_t kind,
                                     graf_batch_plan_t* plan) {
    return create_plan(B, N_host, M_host, w_host, l_host, losses_per_waveform, kind, nullptr, 0, nullptr, plan);
}

graf_status_t graf_batch_plan_create_scenarios(int32_t S, const int32_t* src_host, int32_t B_src,
                                               const int32_t* N_src_host, const int32_t* M_host,
                                               const graf_window_t* w_host, const graf_loss_t* l_host,
                                               graf_input_t kind, graf_batch_plan_t* plan) {
    if (!src_host) return GRAF_ERR_INVALID_ARG;
    return create_plan(S, nullptr, M_host, w_host, l_host, 1, kind, src_host, B_src, N_src_host, plan);
}

graf_status_t graf_batch_plan_destroy(graf_batch_plan_t P) {
    if (!P) return GRAF_ERR_INVALID_ARG;
    for (Bucket& bk : P->buckets)
        if (bk.d_items) cudaFree(bk.d_items);
    if (P->d_waves) cudaFree(P->d_waves);
    if (P->d_counters) cudaFree(P->d_counters);
    if (P->d_src_entries) cudaFree(P->d_src_entries);
    if (P->d_src_first) cudaFree(P->d_src_first);
    if (P->d_src_off) cudaFree(P->d_src_off);
    delete P;
    return GRAF_OK;
}

size_t graf_batch_workspace_bytes(graf_batch_plan_t P) {
    if (!P) return 0;
    return P->ws_rec + P->ws_scale + P->ws_csum + P->ws_gpart + P->ws_usum + P->ws_scratch;
}

graf_status_t graf_batch_plan_info(graf_batch_plan_t P, int32_t* n_buckets, int32_t* M_out,
                                   int32_t* rows_per_tile_out, int32_t* items_out, int32_t* fused_out,
                                   int32_t capacity) {
    if (!P || !n_buckets) return GRAF_ERR_INVALID_ARG;
    *n_buckets = (int32_t)P->buckets.size();
    for (int i = 0; i < (int)P->buckets.size() && i < capacity; ++i) {
        const Bucket& bk = P->buckets[i];
        if (M_out) M_out[i] = bk.M;
        if (rows_per_tile_out) rows_per_tile_out[i] = bk.rps * graf::slots_of(bk.M);
        if (items_out) items_out[i] = (int32_t)bk.items.size();
        if (fused_out) fused_out[i] = bk.fused ? 1 : 0;
    }
    return GRAF_OK;
}

static graf_status_t check_ws(graf_batch_plan_t P, void* workspace, size_t workspace_bytes) {
    if (!workspace || workspace_bytes < graf_batch_workspace_bytes(P)) return GRAF_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return GRAF_ERR_WORKSPACE;
    return GRAF_OK;
}

graf_status_t graf_batch_loss_backward(graf_batch_plan_t P, const float* phi, float* out8, const float* dL,
                                       float* grad_phi, void* workspace, size_t workspace_bytes,
                                       void* stream) {
    if (!P || !phi || !out8 || !grad_phi) return GRAF_ERR_INVALID_ARG;
    if (P->kind != GRAF_IN_PHASE) return GRAF_ERR_INVALID_ARG;
    const graf_status_t s = check_ws(P, workspace, workspace_bytes);
    if (s != GRAF_OK) return s;
    return batch_step(P, phi, out8, dL, nullptr, grad_phi, workspace, static_cast<cudaStream_t>(stream));
}

graf_status_t graf_batch_loss_backward_complex(graf_batch_plan_t P, const graf_c32* s_in, float* out8,
                                               const float* dL, graf_c32* grad_s, void* workspace,
                                               size_t workspace_bytes, void* stream) {
    if (!P || !s_in || !out8 || !grad_s) return GRAF_ERR_INVALID_ARG;
    if (P->kind != GRAF_IN_COMPLEX) return GRAF_ERR_INVALID_ARG;
    const graf_status_t s = check_ws(P, workspace, workspace_bytes);
    if (s != GRAF_OK) return s;
    return batch_step(P, s_in, out8, dL, reinterpret_cast<float2*>(grad_s), nullptr, workspace,
                      static_cast<cudaStream_t>(stream));
}

graf_status_t graf_batch_loss(graf_batch_plan_t P, const void* x, float* out8, void* workspace,
                              size_t workspace_bytes, void* stream) {
    if (!P || !x || !out8) return GRAF_ERR_INVALID_ARG;
    graf_status_t s = check_ws(P, workspace, workspace_bytes);
    if (s != GRAF_OK) return s;
    bool two = false;
    return batch_loss_rows(P, x, out8, workspace, false, &two, static_cast<cudaStream_t>(stream));
}

graf_status_t graf_batch_af_offsets(graf_batch_plan_t P, int64_t* af_off_host) {
    if (!P || !af_off_host) return GRAF_ERR_INVALID_ARG;
    for (size_t i = 0; i < P->af_off.size(); ++i) af_off_host[i] = P->af_off[i];
    return GRAF_OK;
}

graf_status_t graf_batch_forward(graf_batch_plan_t P, const void* x, float* af_out, void* stream) {
    if (!P || !x || !af_out) return GRAF_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (size_t i = 0; i < P->buckets.size(); ++i) {
        const Bucket& bk = P->buckets[i];
        AfParams p = bucket_params(P, bk, (int)i, x, nullptr, nullptr);
        p.af_out = af_out;
        p.chi_out = 0;
        if (cudaMemsetAsync(p.counter, 0, sizeof(unsigned int), st) != cudaSuccess) return GRAF_ERR_CUDA;
        if (graf::run_forward(p, st) != cudaSuccess) return GRAF_ERR_CUDA;
    }
    return GRAF_OK;
}

graf_status_t graf_batch_autotune(graf_batch_plan_t P, const float* phi, float* out8, float* grad_phi,
                                  void* workspace, size_t workspace_bytes, void* stream,
                                  const char* cache_path) {
    if (!P || !phi || !out8 || !grad_phi) return GRAF_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // cached choices: lines "M rps"
    std::vector<std::pair<int, int>> cache;
    if (cache_path) {
        if (FILE* f = std::fopen(cache_path, "r")) {
            int m, r;
            while (std::fscanf(f, "%d %d", &m, &r) == 2) cache.push_back({m, r});
            std::fclose(f);
        }
    }
    const int cand[] = {1, 2, 4, 8, 16};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GRAF_ERR_CUDA;
    graf_status_t s = GRAF_OK;
    for (size_t i = 0; i < P->buckets.size() && s == GRAF_OK; ++i) {
        Bucket& bk = P->buckets[i];
        int best = -1;
        for (auto& c : cache)
            if (c.first == bk.M) best = c.second;
        if (best < 0) {
            float best_ms = 1e30f;
            for (int rps : cand) {
                bk.rps = rps;
                if ((s = layout(P)) != GRAF_OK) break;
                if (workspace_bytes < graf_batch_workspace_bytes(P)) continue;  // too many tiles for the buffer
                const int which = bk.fused ? 0 : 1;
                float ms = 0.0f;
                for (int rep = 0; rep < 3 && s == GRAF_OK; ++rep) {
                    cudaEventRecord(e0, st);
                    s = run_rows(P, bk, (int)i, phi, workspace, out8, which, st);
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    float t = 0.0f;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (rep > 0) ms += t;
                }
                if (s == GRAF_OK && ms < best_ms) {
                    best_ms = ms;
                    best = rps;
                }
            }
            if (best > 0) cache.push_back({bk.M, best});
        }
        if (best > 0) bk.rps = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != GRAF_OK) return s;
    s = layout(P);
    if (s == GRAF_OK && cache_path) {
        if (FILE* f = std::fopen(cache_path, "w")) {
            for (auto& c : cache) std::fprintf(f, "%d %d\n", c.first, c.second);
            std::fclose(f);
        }
    }
    return s;
}

}  // extern "C"
