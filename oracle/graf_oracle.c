/*
 * FP64 CPU oracle for the differentiable discrete ambiguity function.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the bench's CPU-baseline
 * leg use it.  It shares no code, header, table or constant with the CUDA
 * library; every quantity is recomputed here from its definition.
 *
 * Definitions followed (paper section / equation):
 *   - lag product R[k,n] = s[n] * conj(s[n-k])                 (Sec. 4.1, Eq. 8)
 *     taken aperiodically: s[n] = 0 outside [0, N), delays k = -(N-1)..N-1
 *     (the non-periodic extension that Sec. 8.6 lists among the limitations).
 *   - row DFT X[k,m] = sum_n R[k,n] exp(-j 2 pi m n / M)        (Sec. 4.1, Eq. 11)
 *     with an M-point (zero padded) transform, m in [-M/2, M/2-1] (fftshift
 *     order, as in Algorithm 1).
 *   - eps-stabilised, energy-normalised magnitude
 *     Ahat = sqrt(|X|^2 + eps) / E, E = sum |s|^2             (Eq. 12, Eq. 17;
 *     E equals max |X| = |X[0,0]| by Cauchy-Schwarz).
 *   - losses on the sidelobe region Omega (Eq. 18 PSL, Eq. 19 ISL, Eq. 22):
 *       ISL      = sum_Omega Ahat^2
 *       PSL_soft = (1/beta) log sum_Omega exp(beta Ahat^2)
 *       PSL_hard = max_Omega Ahat^2
 *       L        = w_psl PSL_soft + w_isl ISL   (beta finite)
 *       L        = w_psl PSL_hard + w_isl ISL   (beta = +infinity: the
 *                  hard maximum of Eq. 18, the beta -> infinity limit of
 *                  PSL_soft, with the subgradient through one arg-max cell)
 *   - Wirtinger adjoint (Sec. 3.3 Eq. 6, Sec. 4.2 Eqs. 13-15): the gradient
 *     exported is 2 dL/ds* = dL/dRe(s) + j dL/dIm(s), and for phase input
 *     s = exp(j phi), dL/dphi = 2 Im(dL/ds* . conj(s)).
 *
 * The periodic AF of the paper's own definition (Sec. 3.1 Eq. 2, Sec. 4.1
 * Eq. 7, Algorithm 1) is at the end of the file: circular lag (n - k) mod N,
 * N Doppler bins, exponent sign +j (Eq. 7) or -j (the FFT of Algorithm 1).
 *
 * Every sum is a direct double sum in the order the definition states; no FFT
 * is used anywhere in this file.  Threads only split independent delay rows;
 * partial gradients are added in a fixed order so results are deterministic.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 3

typedef struct {
    int64_t k_lo, k_hi; /* delay window, inclusive */
    int64_t m_lo, m_hi; /* Doppler window, inclusive, fftshift indices */
    int64_t k_ml, m_ml; /* mainlobe box |k|<=k_ml && |m|<=m_ml, excluded from Omega */
} orc_window;

/* ------------------------------------------------------------------ helpers */

static int64_t mod_i64(int64_t a, int64_t m) {
    int64_t r = a % m;
    return r < 0 ? r + m : r;
}

/* W[q] = exp(-j 2 pi q / M) for q in [0, M): the DFT kernel of Eq. 11 with the
 * M-point, negative-exponent convention.  Index (m*n) mod M is exact integer
 * arithmetic, so every twiddle is one double-precision cos/sin of 2 pi q / M. */
static double* make_w_table(int64_t M) {
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)M);
    if (!w) return NULL;
    for (int64_t q = 0; q < M; ++q) {
        double a = 2.0 * ORC_PI * (double)q / (double)M;
        w[2 * q] = cos(a);
        w[2 * q + 1] = -sin(a);
    }
    return w;
}

static int check_window(int64_t N, int64_t M, const orc_window* w) {
    if (N < 1 || M < 1) return ORC_EINVAL;
    if (w->k_lo > w->k_hi || w->m_lo > w->m_hi) return ORC_EINVAL;
    if (w->k_lo < -(N - 1) || w->k_hi > N - 1) return ORC_EINVAL;
    if (w->m_lo < -(M / 2) || w->m_hi > M - 1 - M / 2) return ORC_EINVAL;
    if (w->k_ml < -1 || w->m_ml < -1) return ORC_EINVAL; /* -1: no mainlobe box */
    return ORC_OK;
}

static int in_omega(const orc_window* w, int64_t k, int64_t m) {
    if (k < w->k_lo || k > w->k_hi || m < w->m_lo || m > w->m_hi) return 0;
    int64_t ak = k < 0 ? -k : k, am = m < 0 ? -m : m;
    return !(ak <= w->k_ml && am <= w->m_ml);
}

/* One cell of Eq. 11 on the aperiodic lag product of Eq. 8:
 * X[k,m] = sum_{n} s[n] conj(s[n-k]) W[(m n) mod M], n over the support
 * max(0,k) <= n <= min(N-1, N-1+k). */
static void af_cell(const double* s, int64_t N, int64_t M, const double* W,
                    int64_t k, int64_t m, double* xr, double* xi) {
    int64_t n0 = k > 0 ? k : 0;
    int64_t n1 = k < 0 ? N - 1 + k : N - 1;
    int64_t mm = mod_i64(m, M);
    double ar = 0.0, ai = 0.0;
    for (int64_t n = n0; n <= n1; ++n) {
        double sr = s[2 * n], si = s[2 * n + 1];
        double tr = s[2 * (n - k)], ti = -s[2 * (n - k) + 1]; /* conj(s[n-k]) */
        double rr = sr * tr - si * ti, ri = sr * ti + si * tr;  /* R[k,n] */
        int64_t q = (mm * n) % M;
        double wr = W[2 * q], wi = W[2 * q + 1];
        ar += rr * wr - ri * wi;
        ai += rr * wi + ri * wr;
    }
    *xr = ar;
    *xi = ai;
}

/* ----------------------------------------------------------- thread plumbing */

typedef struct {
    const double* s;
    int64_t N, M;
    const double* W;
    orc_window win;
    int64_t ncols;
    int64_t row_begin, row_end; /* rows of the window, relative to k_lo */
    double* X;                  /* [rows][ncols][2] */
} af_job;

static void* af_worker(void* p) {
    af_job* j = (af_job*)p;
    for (int64_t r = j->row_begin; r < j->row_end; ++r) {
        int64_t k = j->win.k_lo + r;
        for (int64_t c = 0; c < j->ncols; ++c) {
            int64_t m = j->win.m_lo + c;
            double* o = j->X + 2 * (r * j->ncols + c);
            af_cell(j->s, j->N, j->M, j->W, k, m, &o[0], &o[1]);
        }
    }
    return NULL;
}

static int clamp_threads(int nthreads, int64_t rows) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > rows) nthreads = (int)(rows > 0 ? rows : 1);
    return nthreads;
}

/* ------------------------------------------------------------------ public */

/* s[n] = cos(phi[n]) + j sin(phi[n]): unit-modulus phase code (Sec. 7.1.2). */
void orc_signal_from_phase(const double* phi, int64_t N, double* s) {
    for (int64_t n = 0; n < N; ++n) {
        s[2 * n] = cos(phi[n]);
        s[2 * n + 1] = sin(phi[n]);
    }
}

/* E = sum_n |s[n]|^2, the normaliser that replaces max chi (Eq. 17). */
double orc_energy(const double* s, int64_t N) {
    double e = 0.0;
    for (int64_t n = 0; n < N; ++n) e += s[2 * n] * s[2 * n] + s[2 * n + 1] * s[2 * n + 1];
    return e;
}

/* Complex AF X[k,m] over a window, row-major [k_hi-k_lo+1][m_hi-m_lo+1][2]. */
int orc_af_complex(const double* s, int64_t N, int64_t M, int64_t k_lo, int64_t k_hi,
                   int64_t m_lo, int64_t m_hi, double* X, int nthreads) {
    orc_window win = {k_lo, k_hi, m_lo, m_hi, 0, 0};
    if (check_window(N, M, &win)) return ORC_EINVAL;
    double* W = make_w_table(M);
    if (!W) return ORC_ENOMEM;
    int64_t rows = k_hi - k_lo + 1, ncols = m_hi - m_lo + 1;
    nthreads = clamp_threads(nthreads, rows);
    af_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (af_job){s, N, M, W, win, ncols, rows * t / nthreads, rows * (t + 1) / nthreads, X};
        if (t > 0) pthread_create(&th[t], NULL, af_worker, &jobs[t]);
    }
    af_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(W);
    return ORC_OK;
}

/* Ahat[k,m] = sqrt(|X[k,m]|^2 + eps) / E over a window (Eq. 12, Eq. 17). */
int orc_af_ahat(const double* s, int64_t N, int64_t M, int64_t k_lo, int64_t k_hi,
                int64_t m_lo, int64_t m_hi, double eps, double* Ahat, int nthreads) {
    int64_t cells = (k_hi - k_lo + 1) * (m_hi - m_lo + 1);
    if (cells <= 0) return ORC_EINVAL;
    double* X = (double*)malloc(sizeof(double) * 2 * (size_t)cells);
    if (!X) return ORC_ENOMEM;
    int st = orc_af_complex(s, N, M, k_lo, k_hi, m_lo, m_hi, X, nthreads);
    if (st) { free(X); return st; }
    double E = orc_energy(s, N);
    for (int64_t i = 0; i < cells; ++i)
        Ahat[i] = sqrt(X[2 * i] * X[2 * i] + X[2 * i + 1] * X[2 * i + 1] + eps) / E;
    free(X);
    return ORC_OK;
}

/* Selected cells one by one: Ahat at (ks[i], ms[i]).  Used to check full-size
 * GPU outputs at sampled positions. */
int orc_af_cells(const double* s, int64_t N, int64_t M, int64_t ncells, const int64_t* ks,
                 const int64_t* ms, double eps, double* Ahat) {
    double* W = make_w_table(M);
    if (!W) return ORC_ENOMEM;
    double E = orc_energy(s, N);
    for (int64_t i = 0; i < ncells; ++i) {
        if (ks[i] < -(N - 1) || ks[i] > N - 1 || ms[i] < -(M / 2) || ms[i] > M - 1 - M / 2) {
            free(W);
            return ORC_EINVAL;
        }
        double xr, xi;
        af_cell(s, N, M, W, ks[i], ms[i], &xr, &xi);
        Ahat[i] = sqrt(xr * xr + xi * xi + eps) / E;
    }
    free(W);
    return ORC_OK;
}

/* Loss scalars over Omega = window minus mainlobe box:
 *   out[0] L = w_psl PSL_soft + w_isl ISL        (Eq. 22, lambda_2 and lambda_3)
 *   out[1] PSL_soft = (1/beta) log sum exp(beta Ahat^2)   (Eq. 18, smoothed max)
 *   out[2] ISL = sum Ahat^2                       (Eq. 19; Ahat^2 = chi/chi(0,0))
 *   out[3] PSL_hard = max Ahat^2                  (Eq. 18)
 *   out[4] E
 *   out[5] |Omega|
 *   out[6] sum_Omega p Ahat^2 with p = exp(beta (Ahat^2 - PSL_soft)), the
 *          softmax-weighted mean that the dL/dE term needs
 *   out[7] 0
 * The log-sum-exp is taken in two passes (max, then shifted sum).
 * beta = +infinity (hard PSL): out[1] = out[3] = out[6] = max Ahat^2 (the
 * limits of PSL_soft and of the softmax-weighted mean as beta grows) and
 * L = w_psl max + w_isl ISL.
 * peak (nullable): the arg-max cell (k, m), the first in row-major window
 * order (k ascending, then m ascending) among the cells of Omega whose Ahat^2
 * is within a relative 1e-12 of the maximum (cells equal in exact arithmetic
 * differ by FP64 rounding; this keeps the choice among them to the order
 * alone); (0, 0) with an empty Omega. */
static int loss_from_X(const double* X, const orc_window* w, double E, double eps,
                       double w_psl, double w_isl, double beta, double out[8], int64_t peak[2]) {
    int64_t ncols = w->m_hi - w->m_lo + 1;
    double isl = 0.0, amax = -INFINITY, count = 0.0;
    int64_t pk = 0, pm = 0;
    for (int64_t k = w->k_lo; k <= w->k_hi; ++k)
        for (int64_t m = w->m_lo; m <= w->m_hi; ++m) {
            if (!in_omega(w, k, m)) continue;
            const double* x = X + 2 * ((k - w->k_lo) * ncols + (m - w->m_lo));
            double a2 = (x[0] * x[0] + x[1] * x[1] + eps) / (E * E);
            isl += a2;
            if (a2 > amax) amax = a2;
            count += 1.0;
        }
    if (count > 0.0) {
        const double thr = amax - 1e-12 * fabs(amax);
        int found = 0;
        for (int64_t k = w->k_lo; k <= w->k_hi && !found; ++k)
            for (int64_t m = w->m_lo; m <= w->m_hi; ++m) {
                if (!in_omega(w, k, m)) continue;
                const double* x = X + 2 * ((k - w->k_lo) * ncols + (m - w->m_lo));
                double a2 = (x[0] * x[0] + x[1] * x[1] + eps) / (E * E);
                if (a2 >= thr) { pk = k; pm = m; found = 1; break; }
            }
    }
    if (peak) { peak[0] = pk; peak[1] = pm; }
    if (count == 0.0) {
        memset(out, 0, sizeof(double) * 8);
        out[4] = E;
        return ORC_OK;
    }
    if (isinf(beta)) {
        out[0] = w_psl * amax + w_isl * isl;
        out[1] = amax;
        out[2] = isl;
        out[3] = amax;
        out[4] = E;
        out[5] = count;
        out[6] = amax;
        out[7] = 0.0;
        return ORC_OK;
    }
    double z = 0.0;
    for (int64_t k = w->k_lo; k <= w->k_hi; ++k)
        for (int64_t m = w->m_lo; m <= w->m_hi; ++m) {
            if (!in_omega(w, k, m)) continue;
            const double* x = X + 2 * ((k - w->k_lo) * ncols + (m - w->m_lo));
            double a2 = (x[0] * x[0] + x[1] * x[1] + eps) / (E * E);
            z += exp(beta * (a2 - amax));
        }
    double psl_soft = amax + log(z) / beta;
    double spa = 0.0;
    for (int64_t k = w->k_lo; k <= w->k_hi; ++k)
        for (int64_t m = w->m_lo; m <= w->m_hi; ++m) {
            if (!in_omega(w, k, m)) continue;
            const double* x = X + 2 * ((k - w->k_lo) * ncols + (m - w->m_lo));
            double a2 = (x[0] * x[0] + x[1] * x[1] + eps) / (E * E);
            spa += exp(beta * (a2 - psl_soft)) * a2;
        }
    out[0] = w_psl * psl_soft + w_isl * isl;
    out[1] = psl_soft;
    out[2] = isl;
    out[3] = amax;
    out[4] = E;
    out[5] = count;
    out[6] = spa;
    out[7] = 0.0;
    return ORC_OK;
}

int orc_loss(const double* s, int64_t N, int64_t M, const int64_t win6[6], double w_psl,
             double w_isl, double beta, double eps, double out[8], int nthreads) {
    orc_window w = {win6[0], win6[1], win6[2], win6[3], win6[4], win6[5]};
    if (check_window(N, M, &w) || !(beta > 0.0) || eps < 0.0) return ORC_EINVAL;
    int64_t cells = (w.k_hi - w.k_lo + 1) * (w.m_hi - w.m_lo + 1);
    double* X = (double*)malloc(sizeof(double) * 2 * (size_t)cells);
    if (!X) return ORC_ENOMEM;
    int st = orc_af_complex(s, N, M, w.k_lo, w.k_hi, w.m_lo, w.m_hi, X, nthreads);
    if (!st) st = loss_from_X(X, &w, orc_energy(s, N), eps, w_psl, w_isl, beta, out, NULL);
    free(X);
    return st;
}

/* ------------------------------------------------------------------ adjoint */

typedef struct {
    const double* s;
    int64_t N, M;
    const double* W;
    orc_window win;
    const double* G; /* dL/dX* per window cell, [rows][ncols][2] */
    int64_t row_begin, row_end;
    double* g; /* this thread's partial dL/ds*, [N][2], zero on entry */
} adj_job;

/* For each delay row k of the window:
 *   G_R[k,n] = sum_m G[k,m] conj(W[(m n) mod M])   (adjoint of Eq. 11: the
 *              unnormalised inverse DFT of the linear inverse-transform step
 *              of Sec. 4.2)
 *   and the product rule on R[k,n] = s[n] conj(s[n-k]) (Eq. 8):
 *   dL/ds*[n]   += G_R[k,n] s[n-k]          (through R*[k,n])
 *   dL/ds*[n-k] += conj(G_R[k,n]) s[n]       (through R[k,n]).
 * Derivation: R*[k,n] = conj(s[n]) s[n-k] carries s*[n], so d/ds*[n] of
 * sum G_R R* gives G_R[k,n] s[n-k]; R[k,n] carries s*[n-k] and, L being
 * real, dL/dR = conj(G_R), giving conj(G_R[k,n]) s[n] at index n-k. */
static void* adj_worker(void* p) {
    adj_job* j = (adj_job*)p;
    int64_t N = j->N, M = j->M, ncols = j->win.m_hi - j->win.m_lo + 1;
    const double* s = j->s;
    for (int64_t r = j->row_begin; r < j->row_end; ++r) {
        int64_t k = j->win.k_lo + r;
        int64_t n0 = k > 0 ? k : 0;
        int64_t n1 = k < 0 ? N - 1 + k : N - 1;
        for (int64_t n = n0; n <= n1; ++n) {
            double gr = 0.0, gi = 0.0;
            for (int64_t c = 0; c < ncols; ++c) {
                const double* G = j->G + 2 * (r * ncols + c);
                if (G[0] == 0.0 && G[1] == 0.0) continue;
                int64_t mm = mod_i64(j->win.m_lo + c, M);
                int64_t q = (mm * n) % M;
                double wr = j->W[2 * q], wi = -j->W[2 * q + 1]; /* conj(W) */
                gr += G[0] * wr - G[1] * wi;
                gi += G[0] * wi + G[1] * wr;
            }
            /* term through R*[k,n]: G_R[k,n] * s[n-k] into g[n] */
            double ar = s[2 * (n - k)], ai = s[2 * (n - k) + 1];
            j->g[2 * n] += gr * ar - gi * ai;
            j->g[2 * n + 1] += gr * ai + gi * ar;
            /* term through R[k,n]: conj(G_R[k,n]) * s[n] into g[n-k] */
            double br = s[2 * n], bi = s[2 * n + 1];
            j->g[2 * (n - k)] += gr * br + gi * bi;
            j->g[2 * (n - k) + 1] += gr * bi - gi * br;
        }
    }
    return NULL;
}

/* Gradient of the loss of orc_loss.
 * Cell adjoint (Eqs. 13-14 applied to Ahat^2 = (|X|^2+eps)/E^2):
 *   dL/dAhat^2 = w_isl + w_psl p,  p = exp(beta (Ahat^2 - PSL_soft))
 *   (beta = +infinity: p = 1 at the arg-max cell of loss_from_X, 0 elsewhere:
 *   the subgradient of the hard maximum through that one cell)
 *   G[k,m] = dL/dX*[k,m] = (dL/dAhat^2) X[k,m] / E^2   on Omega, 0 elsewhere.
 * Energy term: dAhat^2/dE = -2 Ahat^2 / E, dE/ds* = s, so
 *   dL/ds* += dLdE * s,  dLdE = -(2/E) (w_isl ISL + w_psl sum_Omega p Ahat^2).
 * Exported: grad_s = 2 dL/ds* (interleaved, may be NULL) and, for phase input,
 * grad_phi[n] = 2 Im(dL/ds*[n] conj(s[n])) (may be NULL). out8 as orc_loss. */
int orc_grad(const double* s, int64_t N, int64_t M, const int64_t win6[6], double w_psl,
             double w_isl, double beta, double eps, double* grad_s, double* grad_phi,
             double out[8], int nthreads) {
    orc_window w = {win6[0], win6[1], win6[2], win6[3], win6[4], win6[5]};
    if (check_window(N, M, &w) || !(beta > 0.0) || eps < 0.0) return ORC_EINVAL;
    int64_t rows = w.k_hi - w.k_lo + 1, ncols = w.m_hi - w.m_lo + 1, cells = rows * ncols;
    double* X = (double*)malloc(sizeof(double) * 2 * (size_t)cells);
    double* W = make_w_table(M);
    if (!X || !W) { free(X); free(W); return ORC_ENOMEM; }
    int st = orc_af_complex(s, N, M, w.k_lo, w.k_hi, w.m_lo, w.m_hi, X, nthreads);
    double E = orc_energy(s, N);
    int64_t peak[2];
    if (!st) st = loss_from_X(X, &w, E, eps, w_psl, w_isl, beta, out, peak);
    if (st) { free(X); free(W); return st; }
    double psl_soft = out[1];
    /* X becomes G in place */
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < ncols; ++c) {
            double* x = X + 2 * (r * ncols + c);
            int64_t k = w.k_lo + r, m = w.m_lo + c;
            if (!in_omega(&w, k, m)) { x[0] = x[1] = 0.0; continue; }
            double a2 = (x[0] * x[0] + x[1] * x[1] + eps) / (E * E);
            double p = isinf(beta) ? ((k == peak[0] && m == peak[1]) ? 1.0 : 0.0)
                                   : exp(beta * (a2 - psl_soft));
            double dl_da2 = w_isl + w_psl * p;
            x[0] *= dl_da2 / (E * E);
            x[1] *= dl_da2 / (E * E);
        }
    nthreads = clamp_threads(nthreads, rows);
    double* gparts = (double*)calloc((size_t)nthreads * 2 * (size_t)N, sizeof(double));
    if (!gparts) { free(X); free(W); return ORC_ENOMEM; }
    adj_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (adj_job){s, N, M, W, w, X, rows * t / nthreads, rows * (t + 1) / nthreads,
                            gparts + (size_t)t * 2 * (size_t)N};
        if (t > 0) pthread_create(&th[t], NULL, adj_worker, &jobs[t]);
    }
    adj_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    double dlde = -(2.0 / E) * (w_isl * out[2] + w_psl * out[6]);
    for (int64_t n = 0; n < N; ++n) {
        double gr = 0.0, gi = 0.0;
        for (int t = 0; t < nthreads; ++t) {
            gr += gparts[(size_t)t * 2 * (size_t)N + 2 * n];
            gi += gparts[(size_t)t * 2 * (size_t)N + 2 * n + 1];
        }
        gr += dlde * s[2 * n];
        gi += dlde * s[2 * n + 1];
        if (grad_s) { grad_s[2 * n] = 2.0 * gr; grad_s[2 * n + 1] = 2.0 * gi; }
        /* Im(g conj(s)) = gi*sr - gr*si */
        if (grad_phi) grad_phi[n] = 2.0 * (gi * s[2 * n] - gr * s[2 * n + 1]);
    }
    free(gparts);
    free(X);
    free(W);
    return ORC_OK;
}

/* The arg-max cell of Ahat^2 over Omega that the hard PSL (beta = +infinity)
 * differentiates through: the first in row-major window order among the
 * cells whose Ahat^2 equals the maximum (see loss_from_X). */
int orc_peak_cell(const double* s, int64_t N, int64_t M, const int64_t win6[6], double eps,
                  int64_t peak[2], int nthreads) {
    orc_window w = {win6[0], win6[1], win6[2], win6[3], win6[4], win6[5]};
    if (check_window(N, M, &w) || eps < 0.0) return ORC_EINVAL;
    int64_t cells = (w.k_hi - w.k_lo + 1) * (w.m_hi - w.m_lo + 1);
    double* X = (double*)malloc(sizeof(double) * 2 * (size_t)cells);
    if (!X) return ORC_ENOMEM;
    double out[8];
    int st = orc_af_complex(s, N, M, w.k_lo, w.k_hi, w.m_lo, w.m_hi, X, nthreads);
    if (!st) st = loss_from_X(X, &w, orc_energy(s, N), eps, 1.0, 0.0, INFINITY, out, peak);
    free(X);
    return st;
}

/* Gradient of one cell's Ahat^2[k,m] = (|X[k,m]|^2 + eps) / E^2 (the term
 * the hard PSL adds, times w_psl): the cell adjoint G = X[k,m] / E^2 at that
 * cell alone, the row adjoint and the two product-rule scatters of adj_worker,
 * and the energy term -(2/E) Ahat^2[k,m] s.  Exported as orc_grad's. */
int orc_cell_grad(const double* s, int64_t N, int64_t M, int64_t k, int64_t m, double eps,
                  double* grad_s, double* grad_phi) {
    orc_window w = {k, k, m, m, -1, -1};
    if (check_window(N, M, &w) || eps < 0.0) return ORC_EINVAL;
    double* W = make_w_table(M);
    double* g = (double*)calloc(2 * (size_t)N, sizeof(double));
    if (!W || !g) { free(W); free(g); return ORC_ENOMEM; }
    double G[2];
    af_cell(s, N, M, W, k, m, &G[0], &G[1]);
    double E = orc_energy(s, N);
    double a2 = (G[0] * G[0] + G[1] * G[1] + eps) / (E * E);
    G[0] /= E * E;
    G[1] /= E * E;
    adj_job job = {s, N, M, W, w, G, 0, 1, g};
    adj_worker(&job);
    double dlde = -(2.0 / E) * a2;
    for (int64_t n = 0; n < N; ++n) {
        double gr = g[2 * n] + dlde * s[2 * n], gi = g[2 * n + 1] + dlde * s[2 * n + 1];
        if (grad_s) { grad_s[2 * n] = 2.0 * gr; grad_s[2 * n + 1] = 2.0 * gi; }
        if (grad_phi) grad_phi[n] = 2.0 * (gi * s[2 * n] - gr * s[2 * n + 1]);
    }
    free(W);
    free(g);
    return ORC_OK;
}

/* Central finite differences of orc_loss's L with respect to phi[p]
 * (s = exp(j phi)).  Step h per coordinate.  Tiny N only. */
int orc_fd_grad_phi(const double* phi, int64_t N, int64_t M, const int64_t win6[6],
                    double w_psl, double w_isl, double beta, double eps, double h,
                    double* grad_phi, int nthreads) {
    double* p = (double*)malloc(sizeof(double) * (size_t)N);
    double* s = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    if (!p || !s) { free(p); free(s); return ORC_ENOMEM; }
    for (int64_t i = 0; i < N; ++i) {
        double o[8], lp, lm;
        memcpy(p, phi, sizeof(double) * (size_t)N);
        p[i] = phi[i] + h;
        orc_signal_from_phase(p, N, s);
        int st = orc_loss(s, N, M, win6, w_psl, w_isl, beta, eps, o, nthreads);
        if (st) { free(p); free(s); return st; }
        lp = o[0];
        p[i] = phi[i] - h;
        orc_signal_from_phase(p, N, s);
        orc_loss(s, N, M, win6, w_psl, w_isl, beta, eps, o, nthreads);
        lm = o[0];
        grad_phi[i] = (lp - lm) / (2.0 * h);
    }
    free(p);
    free(s);
    return ORC_OK;
}

/* Central finite differences with respect to Re s[p] and Im s[p]; the result
 * is dL/dRe + j dL/dIm, interleaved.  Tiny N only. */
int orc_fd_grad_s(const double* s, int64_t N, int64_t M, const int64_t win6[6], double w_psl,
                  double w_isl, double beta, double eps, double h, double* grad_s,
                  int nthreads) {
    double* t = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    if (!t) return ORC_ENOMEM;
    for (int64_t i = 0; i < 2 * N; ++i) {
        double o[8], lp, lm;
        memcpy(t, s, sizeof(double) * 2 * (size_t)N);
        t[i] = s[i] + h;
        int st = orc_loss(t, N, M, win6, w_psl, w_isl, beta, eps, o, nthreads);
        if (st) { free(t); return st; }
        lp = o[0];
        t[i] = s[i] - h;
        orc_loss(t, N, M, win6, w_psl, w_isl, beta, eps, o, nthreads);
        lm = o[0];
        grad_s[i] = (lp - lm) / (2.0 * h);
    }
    free(t);
    return ORC_OK;
}

/* ============================================================ periodic AF */
/* The paper's literal discrete AF (Sec. 3.1 Eq. 2, Sec. 4.1 Eqs. 7-12):
 *   X[k,m] = sum_{n=0}^{N-1} s[n] conj(s[(n-k) mod N]) exp(sign j 2 pi m n / N)
 * with sign = +1 (Eq. 7) or -1 (the forward FFT of Algorithm 1), chi = |X|^2,
 * delays and Doppler bins both in fftshift order k, m in [-N/2, N/2-1]
 * (as in Algorithm 1).  The losses use Ahat^2 = (|X|^2 + eps) / E^2 exactly
 * as for the aperiodic AF; with eps = 0 that is chi / chi[0,0] = chi / max chi
 * (Eq. 17: |X| <= E by Cauchy-Schwarz, with equality at the origin). */

static int check_pwindow(int64_t N, const orc_window* w) {
    if (N < 1) return ORC_EINVAL;
    if (w->k_lo > w->k_hi || w->m_lo > w->m_hi) return ORC_EINVAL;
    if (w->k_lo < -(N / 2) || w->k_hi > N - 1 - N / 2) return ORC_EINVAL;
    if (w->m_lo < -(N / 2) || w->m_hi > N - 1 - N / 2) return ORC_EINVAL;
    if (w->k_ml < -1 || w->m_ml < -1) return ORC_EINVAL;
    return ORC_OK;
}

/* exp(sign j 2 pi q / N) for q in [0, N). */
static double* make_pw_table(int64_t N, int sign) {
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    if (!w) return NULL;
    for (int64_t q = 0; q < N; ++q) {
        double a = 2.0 * ORC_PI * (double)q / (double)N;
        w[2 * q] = cos(a);
        w[2 * q + 1] = sign > 0 ? sin(a) : -sin(a);
    }
    return w;
}

static void paf_cell(const double* s, int64_t N, const double* W, int64_t k, int64_t m,
                     double* xr, double* xi) {
    int64_t mm = mod_i64(m, N);
    double ar = 0.0, ai = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        int64_t j = mod_i64(n - k, N);
        double sr = s[2 * n], si = s[2 * n + 1];
        double tr = s[2 * j], ti = -s[2 * j + 1];              /* conj(s[(n-k) mod N]) */
        double rr = sr * tr - si * ti, ri = sr * ti + si * tr;  /* R[k,n], Eq. 8 */
        int64_t q = (mm * n) % N;
        double wr = W[2 * q], wi = W[2 * q + 1];
        ar += rr * wr - ri * wi;
        ai += rr * wi + ri * wr;
    }
    *xr = ar;
    *xi = ai;
}

/* Complex periodic AF over a window (fftshift coordinates), [rows][cols][2]. */
int orc_paf_complex(const double* s, int64_t N, int sign, int64_t k_lo, int64_t k_hi, int64_t m_lo,
                    int64_t m_hi, double* X) {
    orc_window w = {k_lo, k_hi, m_lo, m_hi, 0, 0};
    if (check_pwindow(N, &w) || (sign != 1 && sign != -1)) return ORC_EINVAL;
    double* W = make_pw_table(N, sign);
    if (!W) return ORC_ENOMEM;
    int64_t ncols = m_hi - m_lo + 1;
    for (int64_t k = k_lo; k <= k_hi; ++k)
        for (int64_t m = m_lo; m <= m_hi; ++m) {
            double* o = X + 2 * ((k - k_lo) * ncols + (m - m_lo));
            paf_cell(s, N, W, k, m, &o[0], &o[1]);
        }
    free(W);
    return ORC_OK;
}

/* Loss scalars of the periodic AF, out8 as orc_loss. */
int orc_ploss(const double* s, int64_t N, int sign, const int64_t win6[6], double w_psl,
              double w_isl, double beta, double eps, double out[8]) {
    orc_window w = {win6[0], win6[1], win6[2], win6[3], win6[4], win6[5]};
    if (check_pwindow(N, &w) || !(beta > 0.0) || eps < 0.0) return ORC_EINVAL;
    int64_t cells = (w.k_hi - w.k_lo + 1) * (w.m_hi - w.m_lo + 1);
    double* X = (double*)malloc(sizeof(double) * 2 * (size_t)cells);
    if (!X) return ORC_ENOMEM;
    int st = orc_paf_complex(s, N, sign, w.k_lo, w.k_hi, w.m_lo, w.m_hi, X);
    if (!st) st = loss_from_X(X, &w, orc_energy(s, N), eps, w_psl, w_isl, beta, out, NULL);
    free(X);
    return st;
}

/* Gradient of orc_ploss: the same cell adjoint and energy term as orc_grad;
 * the row adjoint is G_R[k,n] = sum_m G[k,m] conj(exp(sign j 2 pi m n / N))
 * and the product rule on R[k,n] = s[n] conj(s[(n-k) mod N]) scatters
 *   G_R[k,n] s[(n-k) mod N]  into dL/ds*[n],
 *   conj(G_R[k,n]) s[n]      into dL/ds*[(n-k) mod N]. */
int orc_pgrad(const double* s, int64_t N, int sign, const int64_t win6[6], double w_psl,
              double w_isl, double beta, double eps, double* grad_s, double* grad_phi,
              double out[8]) {
    orc_window w = {win6[0], win6[1], win6[2], win6[3], win6[4], win6[5]};
    if (check_pwindow(N, &w) || !(beta > 0.0) || eps < 0.0) return ORC_EINVAL;
    int64_t rows = w.k_hi - w.k_lo + 1, ncols = w.m_hi - w.m_lo + 1, cells = rows * ncols;
    double* X = (double*)malloc(sizeof(double) * 2 * (size_t)cells);
    double* W = make_pw_table(N, sign);
    double* g = (double*)calloc(2 * (size_t)N, sizeof(double));
    if (!X || !W || !g) { free(X); free(W); free(g); return ORC_ENOMEM; }
    int st = orc_paf_complex(s, N, sign, w.k_lo, w.k_hi, w.m_lo, w.m_hi, X);
    double E = orc_energy(s, N);
    int64_t peak[2];
    if (!st) st = loss_from_X(X, &w, E, eps, w_psl, w_isl, beta, out, peak);
    if (st) { free(X); free(W); free(g); return st; }
    double psl_soft = out[1];
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < ncols; ++c) {
            double* x = X + 2 * (r * ncols + c);
            int64_t k = w.k_lo + r, m = w.m_lo + c;
            if (!in_omega(&w, k, m)) { x[0] = x[1] = 0.0; continue; }
            double a2 = (x[0] * x[0] + x[1] * x[1] + eps) / (E * E);
            double p = isinf(beta) ? ((k == peak[0] && m == peak[1]) ? 1.0 : 0.0)
                                   : exp(beta * (a2 - psl_soft));
            double dl_da2 = w_isl + w_psl * p;
            x[0] *= dl_da2 / (E * E);
            x[1] *= dl_da2 / (E * E);
        }
    for (int64_t r = 0; r < rows; ++r) {
        int64_t k = w.k_lo + r;
        for (int64_t n = 0; n < N; ++n) {
            double gr = 0.0, gi = 0.0;
            for (int64_t c = 0; c < ncols; ++c) {
                const double* G = X + 2 * (r * ncols + c);
                if (G[0] == 0.0 && G[1] == 0.0) continue;
                int64_t q = (mod_i64(w.m_lo + c, N) * n) % N;
                double wr = W[2 * q], wi = -W[2 * q + 1]; /* conj */
                gr += G[0] * wr - G[1] * wi;
                gi += G[0] * wi + G[1] * wr;
            }
            int64_t j = mod_i64(n - k, N);
            double ar = s[2 * j], ai = s[2 * j + 1];
            g[2 * n] += gr * ar - gi * ai;
            g[2 * n + 1] += gr * ai + gi * ar;
            double br = s[2 * n], bi = s[2 * n + 1];
            g[2 * j] += gr * br + gi * bi;
            g[2 * j + 1] += gr * bi - gi * br;
        }
    }
    double dlde = -(2.0 / E) * (w_isl * out[2] + w_psl * out[6]);
    for (int64_t n = 0; n < N; ++n) {
        double gr = g[2 * n] + dlde * s[2 * n], gi = g[2 * n + 1] + dlde * s[2 * n + 1];
        if (grad_s) { grad_s[2 * n] = 2.0 * gr; grad_s[2 * n + 1] = 2.0 * gi; }
        if (grad_phi) grad_phi[n] = 2.0 * (gi * s[2 * n] - gr * s[2 * n + 1]);
    }
    free(X);
    free(W);
    free(g);
    return ORC_OK;
}

/* The arg-max cell of the periodic AF's Ahat^2 over Omega (as orc_peak_cell). */
int orc_ppeak_cell(const double* s, int64_t N, int sign, const int64_t win6[6], double eps, int64_t peak[2]) {
    orc_window w = {win6[0], win6[1], win6[2], win6[3], win6[4], win6[5]};
    if (check_pwindow(N, &w) || eps < 0.0) return ORC_EINVAL;
    int64_t cells = (w.k_hi - w.k_lo + 1) * (w.m_hi - w.m_lo + 1);
    double* X = (double*)malloc(sizeof(double) * 2 * (size_t)cells);
    if (!X) return ORC_ENOMEM;
    double out[8];
    int st = orc_paf_complex(s, N, sign, w.k_lo, w.k_hi, w.m_lo, w.m_hi, X);
    if (!st) st = loss_from_X(X, &w, orc_energy(s, N), eps, 1.0, 0.0, INFINITY, out, peak);
    free(X);
    return st;
}

/* Gradient of one periodic cell's Ahat^2[k,m] = (|X[k,m]|^2 + eps) / E^2:
 * G = X[k,m] / E^2 at that cell, G_R[n] = G conj(exp(sign j 2 pi m n / N)),
 * the product rule on R[k,n] = s[n] conj(s[(n-k) mod N]) as in orc_pgrad, and
 * the energy term -(2/E) Ahat^2 s. */
int orc_pcell_grad(const double* s, int64_t N, int sign, int64_t k, int64_t m, double eps, double* grad_s,
                   double* grad_phi) {
    orc_window w = {k, k, m, m, -1, -1};
    if (check_pwindow(N, &w) || (sign != 1 && sign != -1) || eps < 0.0) return ORC_EINVAL;
    double* W = make_pw_table(N, sign);
    double* g = (double*)calloc(2 * (size_t)N, sizeof(double));
    if (!W || !g) { free(W); free(g); return ORC_ENOMEM; }
    double G[2];
    paf_cell(s, N, W, k, m, &G[0], &G[1]);
    double E = orc_energy(s, N);
    double a2 = (G[0] * G[0] + G[1] * G[1] + eps) / (E * E);
    G[0] /= E * E;
    G[1] /= E * E;
    for (int64_t n = 0; n < N; ++n) {
        int64_t q = (mod_i64(m, N) * n) % N;
        double wr = W[2 * q], wi = -W[2 * q + 1]; /* conj */
        double gr = G[0] * wr - G[1] * wi, gi = G[0] * wi + G[1] * wr;
        int64_t j = mod_i64(n - k, N);
        double ar = s[2 * j], ai = s[2 * j + 1];
        g[2 * n] += gr * ar - gi * ai;
        g[2 * n + 1] += gr * ai + gi * ar;
        double br = s[2 * n], bi = s[2 * n + 1];
        g[2 * j] += gr * br + gi * bi;
        g[2 * j + 1] += gr * bi - gi * br;
    }
    double dlde = -(2.0 / E) * a2;
    for (int64_t n = 0; n < N; ++n) {
        double gr = g[2 * n] + dlde * s[2 * n], gi = g[2 * n + 1] + dlde * s[2 * n + 1];
        if (grad_s) { grad_s[2 * n] = 2.0 * gr; grad_s[2 * n + 1] = 2.0 * gi; }
        if (grad_phi) grad_phi[n] = 2.0 * (gi * s[2 * n] - gr * s[2 * n + 1]);
    }
    free(W);
    free(g);
    return ORC_OK;
}

/* Central finite differences of orc_ploss's L with respect to phi[p]. */
int orc_pfd_grad_phi(const double* phi, int64_t N, int sign, const int64_t win6[6], double w_psl,
                     double w_isl, double beta, double eps, double h, double* grad_phi) {
    double* p = (double*)malloc(sizeof(double) * (size_t)N);
    double* s = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    if (!p || !s) { free(p); free(s); return ORC_ENOMEM; }
    for (int64_t i = 0; i < N; ++i) {
        double o[8], lp, lm;
        memcpy(p, phi, sizeof(double) * (size_t)N);
        p[i] = phi[i] + h;
        orc_signal_from_phase(p, N, s);
        int st = orc_ploss(s, N, sign, win6, w_psl, w_isl, beta, eps, o);
        if (st) { free(p); free(s); return st; }
        lp = o[0];
        p[i] = phi[i] - h;
        orc_signal_from_phase(p, N, s);
        orc_ploss(s, N, sign, win6, w_psl, w_isl, beta, eps, o);
        lm = o[0];
        grad_phi[i] = (lp - lm) / (2.0 * h);
    }
    free(p);
    free(s);
    return ORC_OK;
}

/* ============================================================ match term */
/* L_match = weight * sum_window (Ahat^2[k,m] - target[k,m])^2 (Sec. 5.2,
 * Eq. 22, on Ahat^2 = (|X|^2 + eps) / E^2), target laid out [rows][cols] over
 * the window.  Gradient by the same direct adjoint as orc_grad with the cell
 * adjoint dL/dAhat^2 = 2 weight (Ahat^2 - target) and the energy term
 * dL/dE = -(2/E) sum dL/dAhat^2 Ahat^2.  out[0] = the unweighted sum. */
int orc_match(const double* s, int64_t N, int64_t M, const int64_t win6[6], const double* target,
              double weight, double eps, double* grad_s, double* grad_phi, double out[1], int nthreads) {
    orc_window w = {win6[0], win6[1], win6[2], win6[3], -1, -1};
    if (check_window(N, M, &w) || eps < 0.0) return ORC_EINVAL;
    int64_t rows = w.k_hi - w.k_lo + 1, ncols = w.m_hi - w.m_lo + 1, cells = rows * ncols;
    double* X = (double*)malloc(sizeof(double) * 2 * (size_t)cells);
    double* W = make_w_table(M);
    if (!X || !W) { free(X); free(W); return ORC_ENOMEM; }
    int st = orc_af_complex(s, N, M, w.k_lo, w.k_hi, w.m_lo, w.m_hi, X, nthreads);
    if (st) { free(X); free(W); return st; }
    double E = orc_energy(s, N);
    double loss = 0.0, de = 0.0;
    for (int64_t i = 0; i < cells; ++i) {
        double* x = X + 2 * i;
        double a2 = (x[0] * x[0] + x[1] * x[1] + eps) / (E * E);
        double d = a2 - target[i];
        loss += d * d;
        double dl = 2.0 * weight * d;
        de += dl * a2;
        x[0] *= dl / (E * E);
        x[1] *= dl / (E * E);
    }
    out[0] = loss;
    if (grad_s || grad_phi) {
        nthreads = clamp_threads(nthreads, rows);
        double* gparts = (double*)calloc((size_t)nthreads * 2 * (size_t)N, sizeof(double));
        if (!gparts) { free(X); free(W); return ORC_ENOMEM; }
        adj_job jobs[256];
        pthread_t th[256];
        for (int t = 0; t < nthreads; ++t) {
            jobs[t] = (adj_job){s, N, M, W, w, X, rows * t / nthreads, rows * (t + 1) / nthreads,
                                gparts + (size_t)t * 2 * (size_t)N};
            if (t > 0) pthread_create(&th[t], NULL, adj_worker, &jobs[t]);
        }
        adj_worker(&jobs[0]);
        for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
        double dlde = -(2.0 / E) * de;
        for (int64_t n = 0; n < N; ++n) {
            double gr = dlde * s[2 * n], gi = dlde * s[2 * n + 1];
            for (int t = 0; t < nthreads; ++t) {
                gr += gparts[(size_t)t * 2 * (size_t)N + 2 * n];
                gi += gparts[(size_t)t * 2 * (size_t)N + 2 * n + 1];
            }
            if (grad_s) { grad_s[2 * n] = 2.0 * gr; grad_s[2 * n + 1] = 2.0 * gi; }
            if (grad_phi) grad_phi[n] = 2.0 * (gi * s[2 * n] - gr * s[2 * n + 1]);
        }
        free(gparts);
    }
    free(X);
    free(W);
    return ORC_OK;
}
