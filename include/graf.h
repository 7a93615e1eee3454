/*
 * graf.h - C ABI of the GB300 (sm_103a) differentiable ambiguity-function
 * library: the discrete ambiguity function (AF) of a complex waveform, its
 * fused sidelobe losses and their Wirtinger-calculus gradient.
 *
 * Method: GRAF, from M. Bara, "Differentiable Radar Ambiguity Functions:
 * Mathematical Formulation and Computational Implementation" (arXiv 2506.22935):
 *   lag product   R[k,n] = s[n] conj(s[n-k])                        Sec. 4.1, Eq. 8
 *                 aperiodic: s[n] = 0 outside [0,N), k = -(N-1)..N-1 (the
 *                 non-periodic extension listed in Sec. 8.6); the paper's own
 *                 circular form is the graf_paf_* family at the end
 *   row DFT       X[k,m] = sum_n R[k,n] exp(-2 pi j m n / M)          Sec. 4.1, Eq. 11
 *                 M-point (zero padded), m in [-M/2, M/2-1]         (fftshift, Algorithm 1)
 *   magnitude     Ahat[k,m] = sqrt(|X[k,m]|^2 + eps) / E,           Eq. 12, Eq. 17
 *                 E = sum_n |s[n]|^2 (= max |X| = |X[0,0]|)
 *   losses on the sidelobe region Omega (Eqs. 18, 19, 22):
 *                 ISL = sum_Omega Ahat^2,  PSL_hard = max_Omega Ahat^2,
 *                 PSL_soft = (1/beta) log sum_Omega exp(beta Ahat^2),
 *                 L = w_psl PSL_soft + w_isl ISL  (beta finite), or
 *                 L = w_psl PSL_hard + w_isl ISL  (beta = +infinity: the hard
 *                 maximum of Eq. 18, differentiated through one arg-max cell)
 *   gradient      Wirtinger calculus, Sec. 3.3 Eq. 6 and Sec. 4.2 Eqs. 13-15:
 *                 grad_s = 2 dL/ds* = dL/dRe(s) + j dL/dIm(s) (PyTorch's
 *                 convention) and, for s = exp(j phi), grad_phi = dL/dphi.
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers (cudaMalloc'd or torch CUDA
 *     memory) owned by the caller, unless a comment says "host".  Nothing is
 *     allocated, freed or synchronised inside the compute calls: they only
 *     enqueue kernels on `stream` (a cudaStream_t passed as void*; NULL is the
 *     legacy default stream) and return.
 *   - Batches are B waveforms of equal length N stored contiguously:
 *     GRAF_IN_COMPLEX: graf_c32 x[B][N] (interleaved re, im; complex64);
 *     GRAF_IN_PHASE:   float   x[B][N] phases phi, s[n] = exp(j phi[n]).
 *   - Constraints: 1 <= B <= 2^20, 1 <= N <= M, M a power of two in
 *     [GRAF_M_MIN, GRAF_M_MAX], window inside k in [-(N-1), N-1] and
 *     m in [-M/2, M/2-1] with lo <= hi, mainlobe box sizes >= -1, eps >= 0,
 *     beta > 0.  A violated constraint returns GRAF_ERR_INVALID_ARG before
 *     anything is enqueued.  A kernel launch error returns GRAF_ERR_CUDA.
 *     What only the device can see (a zero or non-finite energy, a
 *     non-finite loss) is recorded in the device error word, read with
 *     graf_get_device_error.
 *   - Results are deterministic: every reduction runs in a fixed order.
 */
#ifndef GRAF_H
#define GRAF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GRAF_API __attribute__((visibility("default")))
#else
#define GRAF_API
#endif

#define GRAF_VERSION 1
#define GRAF_M_MIN 8
#define GRAF_M_MAX 16384
#define GRAF_LOSS_OUT 8 /* floats per waveform in out8 / saved8 */

typedef enum {
    GRAF_OK = 0,
    GRAF_ERR_INVALID_ARG = 1,
    GRAF_ERR_UNSUPPORTED = 2,
    GRAF_ERR_NOMEM = 3,
    GRAF_ERR_CUDA = 4,
    GRAF_ERR_TIMEOUT = 5,
    GRAF_ERR_DEVICE_FLAG = 6,
    GRAF_ERR_WORKSPACE = 7
} graf_status_t;

/* complex64, interleaved; layout-compatible with float2 and torch.complex64 */
typedef struct {
    float re, im;
} graf_c32;

/* Delay/Doppler window (inclusive bounds, Doppler in fftshift order) and the
 * mainlobe box |k| <= k_ml && |m| <= m_ml that the losses exclude; the
 * sidelobe region of Eq. 18 is Omega = window minus box.  A box size of -1
 * excludes nothing. */
typedef struct {
    int32_t k_lo, k_hi;
    int32_t m_lo, m_hi;
    int32_t k_ml, m_ml;
} graf_window_t;

/* Composite loss weights (Eq. 22, lambda_2 = w_psl, lambda_3 = w_isl), the
 * soft-max temperature beta of PSL_soft and the magnitude stabiliser eps.
 * beta = +INFINITY selects the hard PSL of Eq. 18 (the beta -> infinity limit
 * of PSL_soft): the PSL term is max_Omega Ahat^2 and its gradient is that of
 * one arg-max cell's Ahat^2 (a subgradient; cells equal within FP32 rounding
 * are all valid choices, and mirror cells (k, m), (-k, -m) are one function
 * of s, so they give the same gradient).  Batch plans take finite beta only. */
typedef struct {
    float w_psl, w_isl, beta, eps;
} graf_loss_t;

typedef enum { GRAF_IN_COMPLEX = 0, GRAF_IN_PHASE = 1 } graf_input_t;

/* Human-readable name of a status code (static string, never NULL). */
GRAF_API const char* graf_status_string(graf_status_t status);

/* GRAF_VERSION of the loaded library. */
GRAF_API int32_t graf_version(void);

/* Bits of the device error word.  The calls return before their kernels run,
 * so conditions only the device sees are recorded there, per device, by the
 * loss finalisation of every loss call (graf_af_loss, graf_af_loss_backward,
 * graf_paf_*, the batch plans) and of graf_af_match. */
#define GRAF_DEVERR_ENERGY 1u    /* a waveform's energy E = sum |s|^2 was 0 or not finite */
#define GRAF_DEVERR_NONFINITE 2u /* a loss scalar came out not finite (NaN or Inf in the input) */
#define GRAF_DEVERR_TIMEOUT 4u   /* a bounded wait of a tensor-core kernel (the proposal MLP's GEMMs) ran
                                    out: that kernel stopped, freed its tensor memory, and its output is
                                    not valid */

/*
 * graf_get_device_error_word - takes the current device's error word in
 * stream order (read and cleared in one atomic exchange after the work queued
 * on `stream`), waits for it and returns it in *word (0 = nothing raised).
 * The word collects bits from every stream of the device since it was last
 * taken.
 * GRAF_ERR_INVALID_ARG if word is NULL, GRAF_ERR_CUDA if a CUDA call fails.
 */
GRAF_API graf_status_t graf_get_device_error_word(uint32_t* word, void* stream);

/*
 * graf_get_device_error - as graf_get_device_error_word without the bits:
 * GRAF_OK if the word was 0, else GRAF_ERR_DEVICE_FLAG (the word is cleared).
 */
GRAF_API graf_status_t graf_get_device_error(void* stream);

/*
 * graf_af_forward - the energy-normalised AF over a window (Algorithm 1 with
 * the aperiodic lag, Eqs. 8, 11, 12, 17).
 *   x       [B][N] signal (see graf_input_t)
 *   w       window; k_ml / m_ml are ignored here
 *   eps     magnitude stabiliser (>= 0)
 *   af_out  float [B][k_hi-k_lo+1][m_hi-m_lo+1], row = delay k ascending,
 *           column = Doppler m ascending (fftshift order): Ahat[k,m].
 * Every cell of the window is written.
 */
GRAF_API graf_status_t graf_af_forward(const void* x, graf_input_t kind, int32_t B, int32_t N,
                              int32_t M, graf_window_t w, float eps, float* af_out,
                              void* stream);

/*
 * Workspace (device bytes, 256-byte aligned) that graf_af_loss needs for the
 * given shape; 0 only if the arguments are invalid.
 */
GRAF_API size_t graf_af_loss_workspace_bytes(int32_t B, int32_t N, int32_t M, graf_window_t w);

/*
 * graf_af_loss - fused sidelobe losses (Eqs. 18, 19, 22) without writing the
 * AF to memory.
 *   out8  float [B][GRAF_LOSS_OUT]: per waveform
 *         {L, PSL_soft, ISL, PSL_hard, E, |Omega|, S_p, 0}
 *         where S_p = sum_Omega p Ahat^2, p = exp(beta (Ahat^2 - PSL_soft)),
 *         the softmax-weighted term the energy gradient needs.  With beta =
 *         +infinity, PSL_soft and S_p are PSL_hard (their limits).  If Omega
 *         is empty, L = PSL_soft = ISL = PSL_hard = S_p = 0.
 *   workspace  caller-owned scratch of graf_af_loss_workspace_bytes();
 *         too small -> GRAF_ERR_WORKSPACE.  Its contents are overwritten.
 */
GRAF_API graf_status_t graf_af_loss(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t M,
                           graf_window_t w, graf_loss_t l, float* out8, void* workspace,
                           size_t workspace_bytes, void* stream);

/* Workspace bytes for graf_af_backward (and for graf_af_loss_backward). */
GRAF_API size_t graf_af_backward_workspace_bytes(int32_t B, int32_t N, int32_t M, graf_window_t w);

/*
 * graf_af_backward - gradient of L (as defined for graf_af_loss) with respect
 * to the input, by the Wirtinger chain rule of Sec. 4.2 (Eqs. 13-15): cell
 * adjoint dL/dX* = (dL/dAhat^2) X / E^2, the row adjoint of the DFT (an
 * unnormalised inverse DFT), the product rule on R[k,n] = s[n] conj(s[n-k])
 * for both factors, and the energy term dL/dE * s.  The AF rows are
 * recomputed, never stored.
 *   saved8   [B][GRAF_LOSS_OUT] from graf_af_loss on the SAME x, window and
 *            loss (PSL_soft, ISL and S_p are used).  With beta = +infinity
 *            the call locates the arg-max cell itself (one more pass over
 *            the rows) and does not read saved8.
 *   dL       float [B] upstream gradient dOut/dL per waveform, or NULL for 1
 *   grad_s   graf_c32 [B][N] = dL * (dL/dRe s + j dL/dIm s), or NULL
 *   grad_phi float [B][N] = dL * dL/dphi, or NULL; requires GRAF_IN_PHASE
 * At least one of grad_s / grad_phi must be non-NULL.
 */
GRAF_API graf_status_t graf_af_backward(const void* x, graf_input_t kind, int32_t B, int32_t N,
                               int32_t M, graf_window_t w, graf_loss_t l, const float* saved8,
                               const float* dL, graf_c32* grad_s, float* grad_phi,
                               void* workspace, size_t workspace_bytes, void* stream);

/*
 * graf_af_loss_backward - one forward+backward step: graf_af_loss into out8,
 * then graf_af_backward with saved8 = out8, in stream order.  Same arguments
 * and workspace as graf_af_backward.
 */
GRAF_API graf_status_t graf_af_loss_backward(const void* x, graf_input_t kind, int32_t B, int32_t N,
                                    int32_t M, graf_window_t w, graf_loss_t l, float* out8,
                                    const float* dL, graf_c32* grad_s, float* grad_phi,
                                    void* workspace, size_t workspace_bytes, void* stream);

/* Adam hyper-parameters (Kingma & Ba).  The paper's experiments optimise
 * phase codes with Adam at learning rate 0.01 (Sec. 7.1.2); the betas and
 * eps it leaves unstated are taken as 0.9, 0.999, 1e-8. */
typedef struct {
    float lr, beta1, beta2, eps;
} graf_adam_t;

/* Device bytes of the per-optimiser state graf_adam_step needs (a
 * completion counter); zero it once before the first step. */
GRAF_API size_t graf_adam_state_bytes(void);

/*
 * graf_adam_step - one Adam update of x[count] in place (the gradient-descent
 * refinement of Sec. 6.2, Eq. 23, with Adam's moment estimates):
 *   t = *step + 1, m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   x -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
 * then *step = t.  x, m, v, grad: device float[count]; m and v start at
 * zero.  step: device int32 counter (starts at 0); keeping it on the device
 * lets a captured CUDA graph of many steps replay with no host work.  state:
 * graf_adam_state_bytes() of zeroed device memory, returned to zero by every
 * call.  Invalid hyper-parameters or pointers -> GRAF_ERR_INVALID_ARG.
 */
GRAF_API graf_status_t graf_adam_step(float* x, float* m, float* v, const float* grad, int64_t count,
                                      graf_adam_t hp, int32_t* step, void* state, void* stream);

/*
 * graf_record_loss - history[*step][b] = out8[b][0] for b < B if
 * *step < history_len (the loss curve of an optimisation, kept on the device).
 */
GRAF_API graf_status_t graf_record_loss(const float* out8, int32_t B, float* history, int32_t history_len,
                                        const int32_t* step, void* stream);

/*
 * Batches of unequal waveforms (the batch processing of Sec. 4.3, s in
 * C^{B x N}, made ragged): waveform b has its own length N_b, Doppler length
 * M_b, window and loss.  A plan groups the waveforms by M, splits each
 * waveform's delay rows into tiles, and orders the (waveform, tile) work
 * items longest first; each M then runs as one persistent launch whose CTAs
 * claim items from an atomic counter.  Plans own device memory (created and
 * freed here, never in the compute calls).  A plan is made for one input
 * kind: phase codes (GRAF_IN_PHASE, gradient dL/dphi through
 * graf_batch_loss_backward) or complex signals (GRAF_IN_COMPLEX, gradient
 * dL/dRe s + j dL/dIm s through graf_batch_loss_backward_complex); finite
 * beta only (GRAF_ERR_UNSUPPORTED for +inf).
 *   N_host   host int32[B], 1 <= N_b
 *   M_host   host int32[B] (power of two, N_b <= M_b <= GRAF_M_MAX) or NULL
 *            for the next power of two >= 2 N_b
 *   w_host   host graf_window_t[B], or NULL for every delay and Doppler bin
 *            minus the zero-delay mainlobe box |m| < M_b / N_b
 *   l_host   host graf_loss_t[B] if losses_per_waveform, else [1] for all
 *   kind     GRAF_IN_PHASE or GRAF_IN_COMPLEX (else GRAF_ERR_INVALID_ARG)
 * Packed layout: waveform b occupies elements [off_b, off_b + N_b) of the
 * input (float phases or graf_c32 samples) and of the gradient (likewise),
 * off_b = N_0 + ... + N_{b-1}.
 */
typedef struct graf_batch_plan_s* graf_batch_plan_t;

GRAF_API graf_status_t graf_batch_plan_create(int32_t B, const int32_t* N_host, const int32_t* M_host,
                                              const graf_window_t* w_host, const graf_loss_t* l_host,
                                              int32_t losses_per_waveform, graf_input_t kind,
                                              graf_batch_plan_t* plan);

/*
 * graf_batch_plan_create_scenarios - a plan of S entries that score B_src
 * source waveforms, each under several windows and loss weights (the
 * multi-scenario loss of Eq. 24, L_j = sum over the entries b of source j of
 * lambda_b L_b, lambda_b passed as dL[b] to graf_batch_loss_backward).
 *   src_host   host int32[S], 0 <= src_b < B_src: the source of entry b
 *   N_src_host host int32[B_src], 1 <= N_j
 *   M_host, w_host as graf_batch_plan_create, per entry; l_host host
 *   graf_loss_t[S], per entry.
 * graf_batch_loss_backward then reads the packed sources (source j at
 * [off_j, off_j + N_j), off_j = N_0 + ... + N_{j-1}), writes out8 per entry
 * ([S][GRAF_LOSS_OUT]) and grad_phi per SOURCE (packed like the input):
 * the sum over its entries, in ascending entry order, of dL_b dL_b/dphi.
 */
GRAF_API graf_status_t graf_batch_plan_create_scenarios(int32_t S, const int32_t* src_host, int32_t B_src,
                                                        const int32_t* N_src_host, const int32_t* M_host,
                                                        const graf_window_t* w_host, const graf_loss_t* l_host,
                                                        graf_input_t kind, graf_batch_plan_t* plan);

GRAF_API graf_status_t graf_batch_plan_destroy(graf_batch_plan_t plan);

/* Device workspace for graf_batch_loss_backward (changes after autotuning). */
GRAF_API size_t graf_batch_workspace_bytes(graf_batch_plan_t plan);

/* Per M bucket (largest M first, up to `capacity`): M, rows per tile, work
 * items, and 1 if the bucket runs the fused loss + gradient kernel (0: the
 * loss kernel, then the recomputing backward kernel). */
GRAF_API graf_status_t graf_batch_plan_info(graf_batch_plan_t plan, int32_t* n_buckets, int32_t* M_out,
                                            int32_t* rows_per_tile_out, int32_t* items_out,
                                            int32_t* fused_out, int32_t capacity);

/*
 * graf_batch_loss_backward - loss scalars (out8 [B][GRAF_LOSS_OUT], as
 * graf_af_loss) and grad_phi (packed, dL_b * dL/dphi) for every waveform of
 * a phase plan (a complex plan: GRAF_ERR_INVALID_ARG).  dL: device float[B]
 * or NULL for ones.  Enqueues on `stream`, allocates nothing.
 */
GRAF_API graf_status_t graf_batch_loss_backward(graf_batch_plan_t plan, const float* phi, float* out8,
                                                const float* dL, float* grad_phi, void* workspace,
                                                size_t workspace_bytes, void* stream);

/*
 * graf_batch_loss_backward_complex - the same for a complex plan (Sec. 4.3:
 * batched s in C^{B x N}, here ragged): s packed graf_c32, grad_s packed
 * graf_c32 = dL_b (dL/dRe s + j dL/dIm s), the Wirtinger gradient of
 * Sec. 4.2 with the energy term of E = sum |s|^2 (a phase plan:
 * GRAF_ERR_INVALID_ARG).
 */
GRAF_API graf_status_t graf_batch_loss_backward_complex(graf_batch_plan_t plan, const graf_c32* s, float* out8,
                                                        const float* dL, graf_c32* grad_s, void* workspace,
                                                        size_t workspace_bytes, void* stream);

/*
 * graf_batch_loss - the loss scalars alone (out8 [B][GRAF_LOSS_OUT], as
 * graf_af_loss; Eqs. 18, 19, 22) for every waveform of the plan, x packed as
 * the plan's input kind; the AF is not written.  Same workspace as the
 * gradient calls.
 */
GRAF_API graf_status_t graf_batch_loss(graf_batch_plan_t plan, const void* x, float* out8, void* workspace,
                                       size_t workspace_bytes, void* stream);

/*
 * graf_batch_af_offsets - host int64[B + 1]: waveform b's window occupies
 * floats [off_b, off_{b+1}) of graf_batch_forward's output (off_B = total).
 */
GRAF_API graf_status_t graf_batch_af_offsets(graf_batch_plan_t plan, int64_t* af_off_host);

/*
 * graf_batch_forward - Ahat = sqrt(|X|^2 + eps) / E (Algorithm 1 with the
 * aperiodic lag; Eqs. 8, 11, 12, 17) over every waveform's window, eps of its
 * plan loss: waveform b's window at af_out + off_b (graf_batch_af_offsets),
 * row-major [k_hi-k_lo+1][m_hi-m_lo+1] as graf_af_forward.  No workspace.
 */
GRAF_API graf_status_t graf_batch_forward(graf_batch_plan_t plan, const void* x, float* af_out, void* stream);

/*
 * graf_batch_autotune - for every M of the plan, time the row kernel with
 * tiles of 1, 2, 4, 8 and 16 rows per slot on these inputs and keep the
 * fastest (the load balance of the persistent launch against the per-tile
 * overhead); choices are read from and written to `cache_path` ("M rows"
 * per line) when it is not NULL.  Synchronises `stream`.  Re-query
 * graf_batch_workspace_bytes afterwards.  Candidates needing more workspace
 * than given are skipped.
 */
GRAF_API graf_status_t graf_batch_autotune(graf_batch_plan_t plan, const float* phi, float* out8,
                                           float* grad_phi, void* workspace, size_t workspace_bytes,
                                           void* stream, const char* cache_path);

/*
 * Learned proposal network (the NN -> waveform -> GRAF -> loss pipeline of
 * Sec. 6.1): an MLP spec[8] -> 512 -> 512 -> 1024 phases, GELU on the hidden
 * layers, BF16 weights on the tensor cores with FP32 accumulation, FP32
 * master weights.  Parameter layout (fp32 master and bf16 copy alike, the
 * bf16 biases unused): W1 [16][512] (rows 8..15 multiply the zero padding
 * of the 8 inputs to the 16-wide MMA k-step) | b1 [512] | W2 [512][512] |
 * b2 [512] | W3 [512][1024] | b3 [1024].  All pointers are device memory.
 */
#define GRAF_MLP_IN 8
#define GRAF_MLP_IN_PAD 16
#define GRAF_MLP_HID 512
#define GRAF_MLP_OUT 1024

/* Number of parameters (floats in the master copy, bf16 in the copy). */
GRAF_API size_t graf_mlp_param_count(void);
/* Bytes of the per-call activation buffer for `rows` specs. */
GRAF_API size_t graf_mlp_activation_bytes(int32_t rows);
/* params_bf16 = bf16(master), round to nearest even. */
GRAF_API graf_status_t graf_mlp_cast_params(const float* master, void* params_bf16, void* stream);
/* phases [rows][1024] fp32 = MLP(spec [rows][8] fp32); keeps what the
 * backward needs in `activations`. */
GRAF_API graf_status_t graf_mlp_forward(const float* spec, int32_t rows, const float* master,
                                        const void* params_bf16, float* phases, void* activations,
                                        void* stream);
/* Label loss per row, invariant to a global phase and to conjugation (the
 * symmetries that leave a Doppler-symmetric masked ISL unchanged):
 * L_b = min_{s=+-1} (1 - |mean_n exp(j(phases_n - s target_n))|) -> loss[b]
 * (may be NULL); scale * dL_b/dphases becomes the output gradient. */
GRAF_API graf_status_t graf_mlp_label_loss(const float* phases, const float* target, int32_t rows,
                                           float scale, float* loss, void* activations, void* stream);
/* Use dphases [rows][1024] (e.g. dL/dphi of an AF loss of the proposed
 * codes) as the output gradient instead. */
GRAF_API graf_status_t graf_mlp_set_output_grad(const float* dphases, int32_t rows, void* activations,
                                                void* stream);
/* grad (fp32, parameter layout) = gradient of the summed output-gradient
 * objective w.r.t. the parameters, for the last forward's activations. */
GRAF_API graf_status_t graf_mlp_backward(int32_t rows, const float* master, const void* params_bf16,
                                         void* activations, float* grad, void* stream);

/*
 * graf_af_loss_backward_noalloc - graf_af_loss_backward without a caller
 * workspace, for callers that cannot allocate device memory (a processing
 * loop whose memory map is fixed at start-up, a host framework whose pool
 * owns all device memory and lends none to plug-ins, code that cannot take
 * cudaMalloc's device synchronisation).  The paper has no counterpart: it is
 * an integration aid of this library.
 *   Arguments and results as graf_af_loss_backward, minus the workspace.
 *   Scratch: a fixed device array of GRAF_NOALLOC_SCRATCH_BYTES (64 MiB)
 *   inside the library, present on every GPU that loads it until the process
 *   exits.  A shape whose graf_af_backward_workspace_bytes() exceeds it
 *   returns GRAF_ERR_WORKSPACE; invalid arguments return
 *   GRAF_ERR_INVALID_ARG.  Nothing is allocated or freed.
 *   Every call looks up the array's device address (cudaGetSymbolAddress)
 *   in the context current at the call, so it stays right after a device
 *   reset and under a caller-created context; the first call in a context
 *   also loads the library's module there, so make that first call before
 *   any stream capture.
 *   All calls share the one array and it keeps the last call's contents:
 *   calls that can overlap on the GPU (different streams, or several host
 *   threads) race on it and must be serialised by the caller.
 */
#define GRAF_NOALLOC_SCRATCH_BYTES (64u << 20)
GRAF_API graf_status_t graf_af_loss_backward_noalloc(const void* x, graf_input_t kind, int32_t B,
                                                     int32_t N, int32_t M, graf_window_t w,
                                                     graf_loss_t l, float* out8, const float* dL,
                                                     graf_c32* grad_s, float* grad_phi, void* stream);

/*
 * Periodic AF: the paper's own discrete definition (Sec. 3.1 Eq. 2, Sec. 4.1
 * Eqs. 7-12, Algorithm 1):
 *   X[k,m] = sum_{n=0}^{N-1} s[n] conj(s[(n-k) mod N]) exp(sign 2 pi j m n / N)
 *   chi[k,m] = |X[k,m]|^2,  k, m in [-N/2, N/2-1] (fftshift order, as in
 *   Algorithm 1),  sign = +1 as in Eq. 7 or -1 as the forward FFT of Algorithm 1.
 * Constraints as above with M = N: N a power of two in [GRAF_M_MIN,
 * GRAF_M_MAX]; windows inside k, m in [-N/2, N/2-1]; sign = +1 or -1, else
 * GRAF_ERR_INVALID_ARG.  The losses are those of the aperiodic calls with
 * Ahat^2 = (|X|^2 + eps) / E^2 (= chi / max chi for eps = 0, Eq. 17) over the
 * window minus the mainlobe box, and so are out8, dL, grad_s and grad_phi.
 */

/* chi_out [B][N][N] (row = delay k ascending, column = Doppler m ascending):
 * chi / E^2 = chi / chi[0,0] = chi / max chi if normalise != 0 (Eq. 17),
 * else chi itself. */
GRAF_API graf_status_t graf_paf_forward(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t sign,
                                        int32_t normalise, float* chi_out, void* stream);
/* Workspace bytes for graf_paf_loss and graf_paf_loss_backward (0 = invalid
 * shape or window). */
GRAF_API size_t graf_paf_workspace_bytes(int32_t B, int32_t N, graf_window_t w);
/* Loss scalars out8 [B][8] as graf_af_loss. */
GRAF_API graf_status_t graf_paf_loss(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t sign,
                                     graf_window_t w, graf_loss_t l, float* out8, void* workspace,
                                     size_t workspace_bytes, void* stream);
/* Loss scalars and gradients as graf_af_loss_backward. */
GRAF_API graf_status_t graf_paf_loss_backward(const void* x, graf_input_t kind, int32_t B, int32_t N,
                                              int32_t sign, graf_window_t w, graf_loss_t l, float* out8,
                                              const float* dL, graf_c32* grad_s, float* grad_phi,
                                              void* workspace, size_t workspace_bytes, void* stream);

/*
 * Spectral variance: the LPI term of the paper's experiment loss (Sec. 7.1.1,
 * Eq. 25), SV = var{|FFT(s)|^2 / sum |FFT(s)|^2} (population variance over the
 * N bins of the N-point DFT), per waveform, and its gradient, so that
 * L = PSL + lambda alpha SV is one graf_paf_loss_backward (or
 * graf_af_loss_backward) followed by this call on the same stream.
 *   x, kind, B, N: as above; N a power of two in [GRAF_M_MIN, GRAF_M_MAX].
 *   weight: lambda alpha.
 *   out8 [B][8] (nullable): out8[b][0] += weight * SV (the total loss) and
 *     out8[b][7] = SV.
 *   sv_out [B] (nullable): SV.
 *   grad_s [B][N] (nullable): weight * 2 dSV/ds*, grad_phi [B][N] (nullable,
 *     phase input only): weight * dSV/dphi; added to the arrays' contents if
 *     accumulate != 0, else written.
 * Errors: GRAF_ERR_INVALID_ARG for a violated constraint, GRAF_ERR_CUDA for a
 * launch failure.
 */
GRAF_API graf_status_t graf_spectral_variance(const void* x, graf_input_t kind, int32_t B, int32_t N,
                                              float weight, float* out8, float* sv_out, graf_c32* grad_s,
                                              float* grad_phi, int32_t accumulate, void* stream);

/*
 * Two more terms of the composite loss (Sec. 5.1 and Sec. 5.2, Eq. 22):
 *   W = sum_{k=-(N-1)}^{N-1} |k| sigmoid(gamma (a2[k] - 1/2)), the
 *       differentiable -3 dB mainlobe width of Sec. 5.1, with
 *       a2[k] = (|r[k]|^2 + eps) / E^2 = chi(k, 0) / chi(0, 0) and
 *       r[k] = sum_n s[n] conj(s[n-k]) the zero-Doppler column of the AF;
 *   V = var(|s|), the constant-modulus penalty L_const of Eq. 22.
 * Adds w_width W + w_const V to out8[b][0] (nullable), writes {W, V} to
 * terms_out [B][2] (nullable), and the gradient of w_width W + w_const V to
 * grad_s [B][N] (2 dL/ds*) or grad_phi [B][N] (phase input), added to their
 * contents if accumulate != 0, else written; N <= GRAF_M_MAX / 2, gamma > 0,
 * eps >= 0 (GRAF_ERR_INVALID_ARG otherwise).  Computed with transforms of
 * length nextpow2(2N), so the lags do not wrap.
 */
GRAF_API graf_status_t graf_composite_terms(const void* x, graf_input_t kind, int32_t B, int32_t N,
                                            float gamma, float eps, float w_width, float w_const, float* out8,
                                            float* terms_out, graf_c32* grad_s, float* grad_phi,
                                            int32_t accumulate, void* stream);

/*
 * graf_af_match - the target-matching term of the composite loss (Sec. 5.2,
 * Eq. 22), L_match = weight * sum over the window of (Ahat^2[k,m] -
 * target[k,m])^2 with Ahat^2 = (|X|^2 + eps) / E^2 = chi / chi(0,0), and its
 * gradient.
 *   target   device float[B][k_hi-k_lo+1][m_hi-m_lo+1], the designer's
 *            reference surface in the layout of graf_af_forward's output,
 *            in units of Ahat^2.
 *   loss_out device float[B] (nullable): sum (Ahat^2 - target)^2, unweighted;
 *   out8     device float[B][8] (nullable): out8[b][0] += weight * that sum;
 *   grad_s / grad_phi as graf_af_backward, for weight * the sum, added to the
 *   arrays' contents if accumulate != 0, else written (both may be NULL).
 * Workspace from graf_af_match_workspace_bytes (256-byte aligned).  Errors
 * as graf_af_backward.
 */
GRAF_API size_t graf_af_match_workspace_bytes(int32_t B, int32_t N, int32_t M, graf_window_t w);
GRAF_API graf_status_t graf_af_match(const void* x, graf_input_t kind, int32_t B, int32_t N, int32_t M,
                                     graf_window_t w, const float* target, float weight, float eps,
                                     float* loss_out, float* out8, graf_c32* grad_s, float* grad_phi,
                                     int32_t accumulate, void* workspace, size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GRAF_H */
