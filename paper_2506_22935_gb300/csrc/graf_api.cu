// graf_api.cu - the C ABI declared in include/graf.h: argument checks,
// workspace layout and kernel launches.  No allocation, no host sync.
#include <cuda_runtime.h>

#include "graf.h"
#include "graf_kernels.cuh"

using graf::AfParams;
using graf::Tiling;

namespace {

bool is_pow2(int32_t v) { return v > 0 && (v & (v - 1)) == 0; }

graf_status_t check_shape(int32_t B, int32_t N, int32_t M) {
    if (B < 1 || B > (1 << 20)) return GRAF_ERR_INVALID_ARG;
    if (!is_pow2(M) || M < GRAF_M_MIN || M > GRAF_M_MAX) return GRAF_ERR_INVALID_ARG;
    if (N < 1 || N > M) return GRAF_ERR_INVALID_ARG;
    return GRAF_OK;
}

// Which AF a call computes: the aperiodic AF (2N-1 delays, M Doppler bins) or
// the periodic AF of Eq. 7 (circular lag, M = N, delays and Doppler bins in
// [-N/2, N/2-1]), the latter with the +j exponent of Eq. 7 (pconj) or -j.
struct Mode {
    int periodic, pconj;
};
constexpr Mode kAperiodic{0, 0};

// shared-memory length of the signal and of each accumulator
int32_t store_len(const Mode& md, int32_t N) { return md.periodic ? 2 * N : N; }

graf_status_t check_window(int32_t N, int32_t M, const graf_window_t& w, const Mode& md = kAperiodic) {
    if (w.k_lo > w.k_hi || w.m_lo > w.m_hi) return GRAF_ERR_INVALID_ARG;
    if (md.periodic) {
        if (w.k_lo < -(N / 2) || w.k_hi > N / 2 - 1) return GRAF_ERR_INVALID_ARG;
    } else if (w.k_lo < -(N - 1) || w.k_hi > N - 1) {
        return GRAF_ERR_INVALID_ARG;
    }
    if (w.m_lo < -(M / 2) || w.m_hi > M / 2 - 1) return GRAF_ERR_INVALID_ARG;
    if (w.k_ml < -1 || w.m_ml < -1) return GRAF_ERR_INVALID_ARG;
    return GRAF_OK;
}

// beta > 0 finite (soft PSL) or +infinity (hard PSL), eps >= 0 finite.
graf_status_t check_loss(const graf_loss_t& l) {
    if (!(l.beta > 0.0f) || !(l.eps >= 0.0f)) return GRAF_ERR_INVALID_ARG;
    if (!(l.w_psl == l.w_psl) || !(l.w_isl == l.w_isl)) return GRAF_ERR_INVALID_ARG;
    if ((l.beta > 1e30f && !graf::is_hard_beta(l.beta)) || l.eps > 1e30f) return GRAF_ERR_INVALID_ARG;
    return GRAF_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

AfParams base_params(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t M,
                     const graf_window_t& w, const Tiling& T, const Mode& md = kAperiodic) {
    AfParams p{};
    p.periodic = md.periodic;
    p.pconj = md.pconj;
    p.x = x;
    p.kind = kind == GRAF_IN_PHASE ? 1 : 0;
    p.B = B; p.N = N; p.M = M;
    p.k_lo = w.k_lo; p.k_hi = w.k_hi; p.m_lo = w.m_lo; p.m_hi = w.m_hi;
    p.k_ml = w.k_ml; p.m_ml = w.m_ml;
    p.r_lo = T.r_lo; p.r_hi = T.r_hi;
    p.rows_per_tile = T.rows_per_tile; p.tiles = T.tiles;
    p.full_m = (w.m_lo == -(M / 2) && w.m_hi == M / 2 - 1) ? 1 : 0;
    return p;
}

graf_status_t cuda_status(cudaError_t e) { return e == cudaSuccess ? GRAF_OK : GRAF_ERR_CUDA; }

size_t loss_ws(int32_t B, const Tiling& T) { return align256((size_t)B * T.tiles * sizeof(float4)); }
// backward workspace: gradient partials [B][tiles][N] complex64 | per-CTA
// sums [B][tiles] float | per-waveform FP64 sums [B][2]
size_t gpart_bytes(int32_t B, int32_t N, const Tiling& T) {
    return align256((size_t)B * T.tiles * N * sizeof(float2));
}
size_t csum_bytes(int32_t B, const Tiling& T) { return align256((size_t)B * T.tiles * sizeof(float)); }
size_t backward_ws(int32_t B, int32_t N, const Tiling& T) {
    return gpart_bytes(B, N, T) + csum_bytes(B, T) + align256((size_t)2 * B * sizeof(double));
}

// Fused loss + gradient (graf_af_loss_backward).  PSL path: rows holding
// mainlobe-box cells are deferred to the recomputing backward kernel; the
// ISL-only path fuses every row.  The PSL path needs a window spanning every
// Doppler bin (otherwise no row is uniform and the two-kernel path runs).
struct FusedPlan {
    bool fused;
    Tiling T1;           // all transformed rows
    int defer_hi;        // -1: none
    bool deferred_launch;
    Tiling T2;           // deferred rows that need a gradient
};

FusedPlan fused_plan(int32_t B, int32_t N, int32_t M, const graf_window_t& w, bool psl, bool phase_only) {
    FusedPlan f{};
    const bool full_m = (w.m_lo == -(M / 2) && w.m_hi == M / 2 - 1);
    f.T1 = graf::make_tiling(B, M, w.k_lo, w.k_hi, graf::device_sm_count());
    f.fused = !psl || full_m;
    f.defer_hi = -1;
    f.deferred_launch = false;
    if (f.fused && psl && w.k_ml >= 0 && w.m_ml >= 0 && w.k_ml >= f.T1.r_lo) {
        f.defer_hi = w.k_ml < f.T1.r_hi ? w.k_ml : f.T1.r_hi;
        const int lo = (phase_only && f.T1.r_lo == 0) ? 1 : f.T1.r_lo;  // row 0: no phase gradient
        if (lo <= f.defer_hi) {
            f.deferred_launch = true;
            f.T2 = graf::make_tiling_rows(B, M, lo, f.defer_hi, graf::device_sm_count());
        }
    }
    (void)N;
    return f;
}

// hard PSL: per-waveform peak records, and the loss scalars graf_af_backward
// recomputes for itself
size_t peak_bytes(int32_t B) { return align256((size_t)B * sizeof(int4)); }
size_t out8_bytes(int32_t B) { return align256((size_t)B * GRAF_LOSS_OUT * sizeof(float)); }

size_t fused_ws(int32_t B, int32_t N, const FusedPlan& f) {
    size_t s = loss_ws(B, f.T1) + csum_bytes(B, f.T1) /* scale */ + csum_bytes(B, f.T1) + gpart_bytes(B, N, f.T1);
    if (f.deferred_launch) s += gpart_bytes(B, N, f.T2) + csum_bytes(B, f.T2);
    return s + align256((size_t)2 * B * sizeof(double)) + peak_bytes(B);
}

graf_status_t check_common(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t M,
                           const graf_window_t& w, const Mode& md = kAperiodic) {
    if (!x) return GRAF_ERR_INVALID_ARG;
    if (kind != GRAF_IN_COMPLEX && kind != GRAF_IN_PHASE) return GRAF_ERR_INVALID_ARG;
    graf_status_t s = check_shape(B, N, M);
    if (s != GRAF_OK) return s;
    if (md.periodic && M != N) return GRAF_ERR_INVALID_ARG;
    return check_window(N, M, w, md);
}

}  // namespace

extern "C" {

const char* graf_status_string(graf_status_t status) {
    switch (status) {
        case GRAF_OK: return "GRAF_OK";
        case GRAF_ERR_INVALID_ARG: return "GRAF_ERR_INVALID_ARG: an argument violates a documented constraint";
        case GRAF_ERR_UNSUPPORTED: return "GRAF_ERR_UNSUPPORTED: shape not supported by this build";
        case GRAF_ERR_NOMEM: return "GRAF_ERR_NOMEM: allocation failed";
        case GRAF_ERR_CUDA: return "GRAF_ERR_CUDA: a CUDA runtime call or kernel launch failed";
        case GRAF_ERR_TIMEOUT: return "GRAF_ERR_TIMEOUT: a bounded device wait expired";
        case GRAF_ERR_DEVICE_FLAG: return "GRAF_ERR_DEVICE_FLAG: a kernel raised its error flag";
        case GRAF_ERR_WORKSPACE: return "GRAF_ERR_WORKSPACE: workspace missing or too small";
    }
    return "unknown graf_status_t";
}

int32_t graf_version(void) { return GRAF_VERSION; }

}  // extern "C"

static graf_status_t af_forward_impl(const Mode& md, const void* x, graf_input_t kind, int32_t B, int32_t N,
                                     int32_t M, graf_window_t w, float eps, int chi_out, float* af_out,
                                     void* stream) {
    graf_status_t s = check_common(x, kind, B, N, M, w, md);
    if (s != GRAF_OK) return s;
    if (!af_out || !(eps >= 0.0f) || eps > 1e30f) return GRAF_ERR_INVALID_ARG;
    if (graf::row_kernel_smem(M, store_len(md, N), 0) > graf::kMaxSmem) return GRAF_ERR_UNSUPPORTED;
    const Tiling T = graf::make_tiling(B, M, w.k_lo, w.k_hi, graf::device_sm_count());
    AfParams p = base_params(x, kind, B, N, M, w, T, md);
    p.eps = eps;
    p.chi_out = chi_out;
    p.af_out = af_out;
    return cuda_status(graf::run_forward(p, static_cast<cudaStream_t>(stream)));
}

static size_t loss_ws_impl(const Mode& md, int32_t B, int32_t N, int32_t M, graf_window_t w) {
    if (check_shape(B, N, M) != GRAF_OK || check_window(N, M, w, md) != GRAF_OK) return 0;
    return loss_ws(B, graf::make_tiling(B, M, w.k_lo, w.k_hi, graf::device_sm_count()));
}

static graf_status_t af_loss_impl(const Mode& md, const void* x, graf_input_t kind, int32_t B, int32_t N,
                                  int32_t M, graf_window_t w, graf_loss_t l, float* out8, void* workspace,
                                  size_t workspace_bytes, void* stream) {
    graf_status_t s = check_common(x, kind, B, N, M, w, md);
    if (s != GRAF_OK) return s;
    if ((s = check_loss(l)) != GRAF_OK) return s;
    if (!out8) return GRAF_ERR_INVALID_ARG;
    if (graf::row_kernel_smem(M, store_len(md, N), 0) > graf::kMaxSmem) return GRAF_ERR_UNSUPPORTED;
    const Tiling T = graf::make_tiling(B, M, w.k_lo, w.k_hi, graf::device_sm_count());
    if (!workspace || workspace_bytes < loss_ws(B, T)) return GRAF_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return GRAF_ERR_WORKSPACE;
    AfParams p = base_params(x, kind, B, N, M, w, T, md);
    p.eps = l.eps; p.beta = l.beta; p.w_psl = l.w_psl; p.w_isl = l.w_isl;
    p.rec = static_cast<float4*>(workspace);
    p.out8 = out8;
    return cuda_status(graf::run_loss(p, static_cast<cudaStream_t>(stream)));
}

static size_t backward_ws_impl(const Mode& md, int32_t B, int32_t N, int32_t M, graf_window_t w) {
    if (check_shape(B, N, M) != GRAF_OK || check_window(N, M, w, md) != GRAF_OK) return 0;
    const Tiling T = graf::make_tiling(B, M, w.k_lo, w.k_hi, graf::device_sm_count());
    size_t s = loss_ws(B, T);
    const size_t b = backward_ws(B, N, T);
    if (b > s) s = b;
    // the fused path's needs for any loss weights and gradient outputs
    for (int psl = 0; psl < 2; ++psl)
        for (int po = 0; po < 2; ++po) {
            const size_t f = fused_ws(B, N, fused_plan(B, N, M, w, psl != 0, po != 0));
            if (f > s) s = f;
        }
    // graf_af_backward with the hard PSL runs the fused step on its own loss scalars
    return s + out8_bytes(B);
}

static graf_status_t af_loss_backward_impl(const Mode& md, const void* x, graf_input_t kind, int32_t B,
                                           int32_t N, int32_t M, graf_window_t w, graf_loss_t l, float* out8,
                                           const float* dL, graf_c32* grad_s, float* grad_phi,
                                           void* workspace, size_t workspace_bytes, void* stream);

static graf_status_t af_backward_impl(const Mode& md, const void* x, graf_input_t kind, int32_t B, int32_t N,
                                      int32_t M, graf_window_t w, graf_loss_t l, const float* saved8,
                                      const float* dL, graf_c32* grad_s, float* grad_phi, void* workspace,
                                      size_t workspace_bytes, void* stream) {
    graf_status_t s = check_common(x, kind, B, N, M, w, md);
    if (s != GRAF_OK) return s;
    if ((s = check_loss(l)) != GRAF_OK) return s;
    if (!saved8 || (!grad_s && !grad_phi)) return GRAF_ERR_INVALID_ARG;
    if (grad_phi && kind != GRAF_IN_PHASE) return GRAF_ERR_INVALID_ARG;
    if (graf::is_hard_beta(l.beta)) {
        // the hard maximum's gradient needs its arg-max cell: run the fused
        // step, with its loss scalars at the end of the workspace
        const size_t need = backward_ws_impl(md, B, N, M, w);
        if (!workspace || workspace_bytes < need) return GRAF_ERR_WORKSPACE;
        if (reinterpret_cast<uintptr_t>(workspace) & 255) return GRAF_ERR_WORKSPACE;
        float* own8 = reinterpret_cast<float*>(static_cast<unsigned char*>(workspace) + need - out8_bytes(B));
        return af_loss_backward_impl(md, x, kind, B, N, M, w, l, own8, dL, grad_s, grad_phi, workspace,
                                     need - out8_bytes(B), stream);
    }
    const Tiling T = graf::make_tiling(B, M, w.k_lo, w.k_hi, graf::device_sm_count());
    if (!workspace || workspace_bytes < backward_ws(B, N, T)) return GRAF_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return GRAF_ERR_WORKSPACE;
    AfParams p = base_params(x, kind, B, N, M, w, T, md);
    p.eps = l.eps; p.beta = l.beta; p.w_psl = l.w_psl; p.w_isl = l.w_isl;
    p.saved8 = saved8;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    p.gpart = reinterpret_cast<float2*>(ws);
    p.csum = reinterpret_cast<float*>(ws + gpart_bytes(B, N, T));
    p.usum = reinterpret_cast<double*>(ws + gpart_bytes(B, N, T) + csum_bytes(B, T));
    p.phase_only = (kind == GRAF_IN_PHASE && grad_s == nullptr) ? 1 : 0;
    p.acc_copies = graf::acc_copies_for(M, N, p.phase_only, md.periodic);
    if (p.acc_copies < 1) return GRAF_ERR_UNSUPPORTED;
    return cuda_status(graf::run_backward(p, dL, reinterpret_cast<float2*>(grad_s), grad_phi,
                                          static_cast<cudaStream_t>(stream)));
}

static graf_status_t af_loss_backward_impl(const Mode& md, const void* x, graf_input_t kind, int32_t B,
                                           int32_t N, int32_t M, graf_window_t w, graf_loss_t l, float* out8,
                                           const float* dL, graf_c32* grad_s, float* grad_phi,
                                           void* workspace, size_t workspace_bytes, void* stream) {
    graf_status_t s = check_common(x, kind, B, N, M, w, md);
    if (s != GRAF_OK) return s;
    if ((s = check_loss(l)) != GRAF_OK) return s;
    if (!out8 || (!grad_s && !grad_phi)) return GRAF_ERR_INVALID_ARG;
    if (grad_phi && kind != GRAF_IN_PHASE) return GRAF_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < backward_ws_impl(md, B, N, M, w) - out8_bytes(B)) return GRAF_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return GRAF_ERR_WORKSPACE;
    const bool phase_only = kind == GRAF_IN_PHASE && grad_s == nullptr;
    const int acc = graf::acc_copies_for(M, N, phase_only ? 1 : 0, md.periodic);
    if (acc < 1) return GRAF_ERR_UNSUPPORTED;
    const bool hard = graf::is_hard_beta(l.beta);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (hard && l.w_isl == 0.0f) {
        // the hard maximum alone: forward transforms with the arg-max cell
        // (loss kernel), the finalisation, then that cell's gradient
        const Tiling T = graf::make_tiling(B, M, w.k_lo, w.k_hi, graf::device_sm_count());
        AfParams p = base_params(x, kind, B, N, M, w, T, md);
        p.eps = l.eps; p.beta = l.beta; p.w_psl = l.w_psl; p.w_isl = l.w_isl;
        p.rec = static_cast<float4*>(workspace);
        p.peak = reinterpret_cast<int4*>(static_cast<unsigned char*>(workspace) + loss_ws(B, T));
        p.out8 = out8;
        cudaError_t e = graf::run_loss(p, st);
        if (e == cudaSuccess)
            e = graf::run_peak_grad(p, dL, reinterpret_cast<float2*>(grad_s), grad_phi, 0, st);
        return cuda_status(e);
    }
    // (hard PSL with ISL: the soft-PSL machinery is off, ISL runs fused, and
    // a loss pass locates the arg-max cell)
    FusedPlan f = fused_plan(B, N, M, w, l.w_psl != 0.0f && !hard, phase_only);
    // on the PSL path with a running log-sum-exp shift each row slot needs its
    // own gradient accumulator (it rescales it); a fixed shift rescales nothing
    const bool fixed = graf::lse_fixed_shift(kind == GRAF_IN_PHASE ? 1 : 0, l.eps, l.beta, N) > 0.0f;
    if (l.w_psl != 0.0f && !hard && !fixed && acc < graf::slots_of(M)) f.fused = false;
    if (!f.fused) {
        s = af_loss_impl(md, x, kind, B, N, M, w, l, out8, workspace, workspace_bytes, stream);
        if (s != GRAF_OK) return s;
        return af_backward_impl(md, x, kind, B, N, M, w, l, out8, dL, grad_s, grad_phi, workspace,
                                workspace_bytes, stream);
    }
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    AfParams p = base_params(x, kind, B, N, M, w, f.T1, md);
    p.eps = l.eps; p.beta = l.beta; p.w_psl = l.w_psl; p.w_isl = l.w_isl;
    p.out8 = out8;
    p.saved8 = out8;
    p.phase_only = phase_only ? 1 : 0;
    p.acc_copies = acc;
    p.defer_hi = f.defer_hi;
    p.rec = reinterpret_cast<float4*>(ws);
    ws += loss_ws(B, f.T1);
    p.scale = reinterpret_cast<float*>(ws);
    ws += csum_bytes(B, f.T1);
    p.csum = reinterpret_cast<float*>(ws);
    ws += csum_bytes(B, f.T1);
    p.gpart = reinterpret_cast<float2*>(ws);
    ws += gpart_bytes(B, N, f.T1);
    float2* gpart2 = nullptr;
    float* csum2 = nullptr;
    if (f.deferred_launch) {
        gpart2 = reinterpret_cast<float2*>(ws);
        ws += gpart_bytes(B, N, f.T2);
        csum2 = reinterpret_cast<float*>(ws);
        ws += csum_bytes(B, f.T2);
    }
    p.usum = reinterpret_cast<double*>(ws);
    ws += align256((size_t)2 * B * sizeof(double));
    if (hard) p.peak = reinterpret_cast<int4*>(ws);
    cudaError_t e = graf::run_fused(p, st);
    // hard PSL: the loss kernel's records (same tiles) carry the arg-max cell;
    // they replace the fused kernel's before the finalisation
    if (e == cudaSuccess) e = hard ? graf::run_loss(p, st) : graf::run_finalize(p, st);
    if (e == cudaSuccess && f.deferred_launch) {
        AfParams q = p;
        q.r_lo = f.T2.r_lo;
        q.r_hi = f.T2.r_hi;
        q.rows_per_tile = f.T2.rows_per_tile;
        q.tiles = f.T2.tiles;
        q.gpart = gpart2;
        q.csum = csum2;
        q.scale = nullptr;
        q.phase_only = 0;  // its rows all need their gradient
        q.acc_copies = graf::acc_copies_for(M, N, 0, md.periodic);  // complex accumulators
        if (q.acc_copies < 1) return GRAF_ERR_UNSUPPORTED;
        e = graf::run_backward(q, nullptr, nullptr, nullptr, st);
        p.tiles2 = f.T2.tiles;
        p.gpart2 = gpart2;
        p.csum2 = csum2;
    }
    if (e == cudaSuccess)
        e = graf::run_grad_reduce(p, dL, reinterpret_cast<float2*>(grad_s), grad_phi, st);
    if (e == cudaSuccess && hard)
        e = graf::run_peak_grad(p, dL, reinterpret_cast<float2*>(grad_s), grad_phi, 1, st);
    return cuda_status(e);
}


extern "C" {

graf_status_t graf_af_forward(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t M,
                              graf_window_t w, float eps, float* af_out, void* stream) {
    return af_forward_impl(kAperiodic, x, kind, B, N, M, w, eps, 0, af_out, stream);
}

size_t graf_af_loss_workspace_bytes(int32_t B, int32_t N, int32_t M, graf_window_t w) {
    return loss_ws_impl(kAperiodic, B, N, M, w);
}

graf_status_t graf_af_loss(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t M,
                           graf_window_t w, graf_loss_t l, float* out8, void* workspace,
                           size_t workspace_bytes, void* stream) {
    return af_loss_impl(kAperiodic, x, kind, B, N, M, w, l, out8, workspace, workspace_bytes, stream);
}

size_t graf_af_backward_workspace_bytes(int32_t B, int32_t N, int32_t M, graf_window_t w) {
    return backward_ws_impl(kAperiodic, B, N, M, w);
}

graf_status_t graf_af_backward(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t M,
                               graf_window_t w, graf_loss_t l, const float* saved8, const float* dL,
                               graf_c32* grad_s, float* grad_phi, void* workspace,
                               size_t workspace_bytes, void* stream) {
    return af_backward_impl(kAperiodic, x, kind, B, N, M, w, l, saved8, dL, grad_s, grad_phi, workspace,
                            workspace_bytes, stream);
}

graf_status_t graf_af_loss_backward(const void* x, graf_input_t kind, int32_t B, int32_t N,
                                    int32_t M, graf_window_t w, graf_loss_t l, float* out8,
                                    const float* dL, graf_c32* grad_s, float* grad_phi,
                                    void* workspace, size_t workspace_bytes, void* stream) {
    return af_loss_backward_impl(kAperiodic, x, kind, B, N, M, w, l, out8, dL, grad_s, grad_phi, workspace,
                                 workspace_bytes, stream);
}

graf_status_t graf_spectral_variance(const void* x, graf_input_t kind, int32_t B, int32_t N, float weight,
                                     float* out8, float* sv_out, graf_c32* grad_s, float* grad_phi,
                                     int32_t accumulate, void* stream) {
    if (!x || (kind != GRAF_IN_COMPLEX && kind != GRAF_IN_PHASE)) return GRAF_ERR_INVALID_ARG;
    if (B < 1 || B > (1 << 20) || !is_pow2(N) || N < GRAF_M_MIN || N > GRAF_M_MAX) return GRAF_ERR_INVALID_ARG;
    if (!(weight == weight) || (grad_phi && kind != GRAF_IN_PHASE)) return GRAF_ERR_INVALID_ARG;
    graf::SpecParams q{};
    q.x = x;
    q.kind = kind == GRAF_IN_PHASE ? 1 : 0;
    q.B = B;
    q.N = N;
    q.weight = weight;
    q.out8 = out8;
    q.sv = sv_out;
    q.grad_s = reinterpret_cast<float2*>(grad_s);
    q.grad_phi = grad_phi;
    q.accumulate = accumulate ? 1 : 0;
    return cuda_status(graf::run_spectral(q, static_cast<cudaStream_t>(stream)));
}

graf_status_t graf_composite_terms(const void* x, graf_input_t kind, int32_t B, int32_t N, float gamma,
                                   float eps, float w_width, float w_const, float* out8, float* terms_out,
                                   graf_c32* grad_s, float* grad_phi, int32_t accumulate, void* stream) {
    if (!x || (kind != GRAF_IN_COMPLEX && kind != GRAF_IN_PHASE)) return GRAF_ERR_INVALID_ARG;
    if (B < 1 || B > (1 << 20) || N < 1 || 2 * N > GRAF_M_MAX) return GRAF_ERR_INVALID_ARG;
    if (!(gamma > 0.0f) || !(eps >= 0.0f) || !(w_width == w_width) || !(w_const == w_const))
        return GRAF_ERR_INVALID_ARG;
    if (grad_phi && kind != GRAF_IN_PHASE) return GRAF_ERR_INVALID_ARG;
    int M = GRAF_M_MIN;
    while (M < 2 * N) M *= 2;
    graf::CompParams q{};
    q.x = x;
    q.kind = kind == GRAF_IN_PHASE ? 1 : 0;
    q.B = B;
    q.N = N;
    q.gamma = gamma;
    q.eps = eps;
    q.w_width = w_width;
    q.w_const = w_const;
    q.out8 = out8;
    q.terms = terms_out;
    q.grad_s = reinterpret_cast<float2*>(grad_s);
    q.grad_phi = grad_phi;
    q.accumulate = accumulate ? 1 : 0;
    return cuda_status(graf::run_composite(q, M, static_cast<cudaStream_t>(stream)));
}

// ------------------------------------------------------------ match term
size_t graf_af_match_workspace_bytes(int32_t B, int32_t N, int32_t M, graf_window_t w) {
    if (check_shape(B, N, M) != GRAF_OK || check_window(N, M, w) != GRAF_OK) return 0;
    const Tiling T = graf::make_tiling(B, M, w.k_lo, w.k_hi, graf::device_sm_count());
    return backward_ws(B, N, T) + csum_bytes(B, T);
}

graf_status_t graf_af_match(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t M, graf_window_t w,
                            const float* target, float weight, float eps, float* loss_out, float* out8,
                            graf_c32* grad_s, float* grad_phi, int32_t accumulate, void* workspace,
                            size_t workspace_bytes, void* stream) {
    graf_status_t s = check_common(x, kind, B, N, M, w);
    if (s != GRAF_OK) return s;
    if (!target || !(weight == weight) || !(eps >= 0.0f) || eps > 1e30f) return GRAF_ERR_INVALID_ARG;
    if (grad_phi && kind != GRAF_IN_PHASE) return GRAF_ERR_INVALID_ARG;
    const Tiling T = graf::make_tiling(B, M, w.k_lo, w.k_hi, graf::device_sm_count());
    if (!workspace || workspace_bytes < graf_af_match_workspace_bytes(B, N, M, w)) return GRAF_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return GRAF_ERR_WORKSPACE;
    const int phase_only = (kind == GRAF_IN_PHASE && grad_s == nullptr) ? 1 : 0;
    const int acc = graf::acc_copies_for(M, N, phase_only);
    if (acc < 1) return GRAF_ERR_UNSUPPORTED;
    AfParams p = base_params(x, kind, B, N, M, w, T);
    p.eps = eps;
    p.beta = 1.0f;  // no log-sum-exp term: w_psl = w_isl = 0
    p.target = target;
    p.match_w = weight;
    p.out8 = out8;
    p.acc_copies = acc;
    p.phase_only = phase_only;
    p.grad_acc = accumulate ? 1 : 0;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    p.gpart = reinterpret_cast<float2*>(ws);
    p.csum = reinterpret_cast<float*>(ws + gpart_bytes(B, N, T));
    p.usum = reinterpret_cast<double*>(ws + gpart_bytes(B, N, T) + csum_bytes(B, T));
    p.mpart = reinterpret_cast<float*>(ws + backward_ws(B, N, T));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = graf::run_match(p, loss_out, st);
    if (e == cudaSuccess && (grad_s || grad_phi))
        e = graf::run_grad_reduce(p, nullptr, reinterpret_cast<float2*>(grad_s), grad_phi, st);
    return cuda_status(e);
}

// ------------------------------------------------------------ periodic AF
static Mode periodic_mode(int32_t sign) { return Mode{1, sign > 0 ? 1 : 0}; }

graf_status_t graf_paf_forward(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t sign,
                               int32_t normalise, float* chi_out, void* stream) {
    if (sign != 1 && sign != -1) return GRAF_ERR_INVALID_ARG;
    const graf_window_t w{-(N / 2), N / 2 - 1, -(N / 2), N / 2 - 1, -1, -1};
    return af_forward_impl(periodic_mode(sign), x, kind, B, N, N, w, 0.0f, normalise ? 1 : 2, chi_out, stream);
}

size_t graf_paf_workspace_bytes(int32_t B, int32_t N, graf_window_t w) {
    return backward_ws_impl(Mode{1, 0}, B, N, N, w);
}

graf_status_t graf_paf_loss(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t sign,
                            graf_window_t w, graf_loss_t l, float* out8, void* workspace,
                            size_t workspace_bytes, void* stream) {
    if (sign != 1 && sign != -1) return GRAF_ERR_INVALID_ARG;
    return af_loss_impl(periodic_mode(sign), x, kind, B, N, N, w, l, out8, workspace, workspace_bytes, stream);
}

graf_status_t graf_paf_loss_backward(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t sign,
                                     graf_window_t w, graf_loss_t l, float* out8, const float* dL,
                                     graf_c32* grad_s, float* grad_phi, void* workspace,
                                     size_t workspace_bytes, void* stream) {
    if (sign != 1 && sign != -1) return GRAF_ERR_INVALID_ARG;
    return af_loss_backward_impl(periodic_mode(sign), x, kind, B, N, N, w, l, out8, dL, grad_s, grad_phi,
                                 workspace, workspace_bytes, stream);
}

}  // extern "C"
