/*
 * lfa.h -- C ABI of the GB300 (sm_103a) library for the singular value
 * decomposition of periodic multi-channel 2-D convolutions by local Fourier
 * analysis (LFA), arXiv 2506.05617: stride-1 layers, and strided layers viewed
 * as crystals (see lfa_layer_desc_t).
 *
 * The method (Sec. III of the paper): a stride-1 convolution on the periodic
 * n x m torus, (A f)(x) = sum_{y in N} M_y f(x + y) with M_y in R^{c_out x c_in}
 * ("Convolutional Mappings"), leaves every Fourier mode invariant. Its SVD is
 * therefore the union, over the n*m frequencies k = (j/n, l/m) of the
 * frequency torus, of the SVDs of the c_out x c_in symbols
 *     A_k = sum_{y in N} M_y exp(2 pi i <k, y>)            ("Convolution Theorem"),
 * and the global singular vectors are the symbol's singular vectors times the
 * Fourier mode (U^_k = F_k^out U_k, V^_k = F_k^in V_k). Algorithm 1 of the
 * paper loops over all frequencies, forms the symbol and takes its SVD; this
 * library does the same on the GPU for all layers of a network at once.
 *
 * Conventions used by every call:
 *  - Weights are float32 in PyTorch's conv layout [c_out][c_in][kh][kw],
 *    row-major, on the device. Tap (a, b) acts at offset
 *    y = (a - pad_h, b - pad_w); pad = -1 selects floor(k/2) (centred stencil,
 *    the paper's 3x3 stencil centred at x). The exponent sign is + as in the
 *    symbol definition above (cross-correlation f(x + y)).
 *  - Rows of the torus are n (frequency index j, tap a, pixel x1); columns are
 *    m (l, b, x2). Frequency f = j*m + l, k = (j/n, l/m).
 *  - r = min(c_out, c_in) singular values per frequency (the thin SVD of the
 *    symbol). The dense operator's remaining |c_out - c_in|*n*m singular
 *    values are exactly zero and are not emitted.
 *  - For real weights A_{-k} = conj(A_k), so only the "half grid" is decomposed:
 *    the frequency f represents the pair {f, fc} with fc = ((n-j)%n)*m + (m-l)%m
 *    when f <= fc. The half grid lists those f in increasing order; its length
 *    is F_h = (n*m + s)/2, s = number of self-conjugate frequencies.
 *  - Complex arrays are interleaved float32 pairs (re, im) ("complex64").
 *  - Singular values are non-negative and sorted in descending order within a
 *    frequency; U and V columns follow the same order.
 *  - Every pointer argument that names GPU data is a device pointer. Arrays of
 *    per-layer pointers ("const float* const* w") are HOST arrays of nlayers
 *    device pointers. The caller owns all input and output buffers; the plan
 *    owns only its own tables and counters.
 *  - Calls that take a stream are asynchronous on that stream (a
 *    cudaStream_t passed as void*; NULL = legacy default stream). Argument
 *    errors are reported synchronously by the return value. Numerical
 *    conditions found on the device (a symbol that did not converge, a
 *    non-finite entry) are counted on the device and read by lfa_get_info().
 *  - No call aborts the process or raises; every failure is a status code.
 *  - A plan is not thread-safe: use one plan per host thread or serialise.
 *  - The calls of one plan share its device workspace (counters, work queue, backward and
 *    log buffers): calls issued on different streams must not overlap on the device. Use
 *    one plan per concurrent stream (e.g. two plans for double-buffered pipelining).
 */
#ifndef LFA_H_
#define LFA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lfa_status {
  LFA_OK = 0,
  LFA_ERR_INVALID_ARG = 1,   /* a size, flag or pointer argument is invalid */
  LFA_ERR_UNSUPPORTED = 2,   /* valid but not supported (e.g. no sm_103 device) */
  LFA_ERR_OOM = 3,           /* a device or pinned-host allocation in lfa_plan failed */
  LFA_ERR_CUDA = 4,          /* a CUDA runtime call failed; see lfa_last_cuda_error() */
  LFA_ERR_NOT_CONVERGED = 5, /* returned by lfa_get_info() when a symbol hit max_sweeps */
  LFA_ERR_NONFINITE = 6,     /* returned by lfa_get_info() when a symbol had NaN/Inf */
  LFA_ERR_TIMEOUT = 7        /* returned by lfa_get_info() when a bounded device wait (the
                                tensor-core route's MMA completion) ran out */
} lfa_status_t;

/* One periodic convolution layer (Sec. III "Convolutional Mappings"):
 * weights [c_out][c_in][kh][kw], tap origin (pad_h, pad_w), -1 = floor(k/2).
 *
 * Stride 1 (stride_h = stride_w = 0 or 1): the layer maps an n x m torus to itself and
 * its symbol A_k is c_out x c_in.
 *
 * Stride (s_h, s_w): the output is (A f)(o, x) = sum_{i,a,b} w[o,i,a,b] f(i, s x + y_ab) on
 * the coarse n x m torus and the input lives on the fine (s_h n) x (s_w m) torus. Viewed as
 * a crystal (Sec. III "Introduction to Lattices and Crystals") the input has s_h s_w points
 * per coarse cell, the polyphase components u = (u_h, u_w) in [0, s_h) x [0, s_w), and the
 * symbol is the c_out x (c_in s_h s_w) matrix
 *   A_k[o][(i, u)] = sum_{taps with y_ab = s q + u} w[o,i,a,b] exp(2 pi i <k, q>),
 * q = floor(y_ab / s) componentwise, column (i, u_h, u_w) at i s_h s_w + u_h s_w + u_w.
 * Everywhere below "c_in" of a symbol, of r and of V then means c_in s_h s_w; the weights
 * and v_hat (which lives on the fine torus, see lfa_expand) keep c_in.
 *
 * Limits: 1 <= c_out <= 512; 1 <= c_in * s_h * s_w <= 512; 1 <= kh, kw <= 15;
 * 1 <= s_h, s_w <= 8; 1 <= n, m <= 65536; n*m <= 2^31 - 1; 0 <= pad < k or -1. */
typedef struct lfa_layer_desc {
  int32_t c_out, c_in, kh, kw, n, m, pad_h, pad_w;
  int32_t stride_h, stride_w;   /* 0 or 1: stride 1 */
} lfa_layer_desc_t;

/* Plan flags. */
#define LFA_VALUES       0x1u  /* singular values (always computed) */
#define LFA_VECTORS      0x2u  /* also the symbol singular vectors U_k, V_k */
#define LFA_HALF_OUTPUT  0x4u  /* sigma only on the half grid, [F_h][r] (else full grid [n*m][r]) */
#define LFA_PLAIN        0x8u  /* plain per-layer path: materialised symbols, one launch per layer
                                  and stage, no graph (the baseline the batched path is measured
                                  against) */
#define LFA_FFT_ROUTE    0x10u /* the plain path with the symbols from the FFT route, the paper's
                                  comparison system (Sec. II, Sec. IV Table II): a batched cuFFT
                                  transform of the zero-padded kernel per channel pair instead of
                                  the tap sums (stride-1 layers, values only; implies LFA_PLAIN) */
#define LFA_REPRODUCIBLE 0x20u /* bitwise identical results from call to call. With vectors the
                                  blocked route (LFA_VARIANT_BLOCKED) normally starts a symbol from
                                  the singular vectors of its neighbouring frequency when that one
                                  is already done, which takes fewer sweeps but depends on timing:
                                  results then differ between calls in rounding (all within the
                                  same tolerance). This flag starts every symbol from W = I
                                  (512 channels: ~12.6 instead of ~8.5 sweeps per symbol). The
                                  other routes are reproducible without it. */

/* Options (nullable pointer: defaults). */
typedef struct lfa_options {
  float tol;            /* one-sided Jacobi threshold: a pair (p, q) is rotated while
                           |x_p^H x_q| > tol * ||x_p|| ||x_q||. <= 0: default
                           max(2^-22, 4 sqrt(M) 2^-24), M = max(c_out, c_in), and at most
                           2^-20 for wide symbols (c_out < c_in), so that A v = sigma u holds
                           to 1e-5 sigma_max for them too */
  int32_t max_sweeps;   /* sweep cap per symbol; <= 0: default 30 */
  int32_t variant;      /* -1: built-in / autotuned choice; >= 0 forces a kernel variant
                           (see lfa_variant_name) for every layer it can run;
                           LFA_VARIANT_LOGGED | v (plans with LFA_VECTORS) runs values-mode
                           variant v with the rotation log, the W replay and the finalize
                           kernel instead of carrying W in registers */
  int32_t use_graph;    /* 1 (default if <0): lfa_svd and lfa_svd_backward replay a CUDA graph
                           captured on their first call with a given set of buffers (the
                           forward's independent kernel groups as parallel branches) */
  const char* tune_cache; /* nullable path of the autotuner's cache (text); read at plan time */
  /* Frequency sharding (the frequencies are independent problems, Algorithm 1; the paper calls
   * LFA embarrassingly parallel, Sec. V). With shard_count = R > 1 every layer's half grid
   * (F_h frequencies, increasing order) is split into R contiguous ranges, range r being
   * [floor(r F_h / R), floor((r + 1) F_h / R)), and the plan decomposes range shard_rank only:
   * one plan per rank (GPU) of a job. F_h, the half-grid list (lfa_layer_query), U, V and the
   * half-grid sigma then cover the shard only ([F_h_shard][...], in the same order); the
   * full-grid sigma layout writes only the shard's frequencies and their conjugates.
   * lfa_svd_backward and lfa_spectral_edit return the shard's contribution (a sum over its
   * frequencies): the job's dL/dw is the sum over ranks (one all-reduce). lfa_expand and
   * lfa_regulariser_grad (whose max term spans all frequencies) return LFA_ERR_UNSUPPORTED on a
   * sharded plan. shard_count <= 1: no sharding (shard_rank must be 0). */
  int32_t shard_rank;
  int32_t shard_count;
} lfa_options_t;

#define LFA_VARIANT_LOGGED 0x10000
/* options.variant value selecting the blocked Jacobi route for every layer it can serve
 * (128 <= N <= 512 columns, M <= 512 rows; not with LFA_PLAIN): one-sided Jacobi over blocks of
 * 32 columns whose Gram matrices and block rotations run on the tcgen05 tensor cores with TF32
 * operands split in three (hi*hi + hi*lo + lo*hi, FP32 accumulation), one CTA per symbol. It is
 * also the built-in choice for tall or square symbols (c_out >= c_in) of more than 128 columns in
 * layers with enough half-grid symbols to fill the GPU (84 up to 256 columns, 30 up to 384, 68 up
 * to 512; fewer go to the element-wise cluster kernels). With vectors a symbol starts from the
 * singular vectors of its neighbouring frequency when that symbol is already done (fewer sweeps;
 * LFA_REPRODUCIBLE turns this off).
 * lfa_layer_query reports it as this value. */
#define LFA_VARIANT_BLOCKED 0x20000

typedef struct lfa_plan_s* lfa_plan_t;

/* Device-side counters of the last lfa_svd on a plan (read by lfa_get_info). */
typedef struct lfa_info {
  int64_t symbols;          /* half-grid symbols decomposed per lfa_svd (all layers) */
  int64_t singular_values;  /* sum over layers of n*m*r (full-grid count) */
  int64_t unconverged;      /* symbols that reached max_sweeps in the last lfa_svd */
  int64_t nonfinite;        /* symbols with a non-finite input or result in the last lfa_svd */
  int64_t sweeps;           /* total sweeps over all symbols in the last lfa_svd */
  int64_t rotations;        /* total applied 2x2 rotations in the last lfa_svd */
  int64_t plan_device_bytes;/* device memory owned by the plan */
  int32_t nlayers;
  int32_t max_sweeps;
  float tol;
  int64_t tc_grams;         /* blocked tensor-core route: block-pair Gram matrices formed */
  int64_t tc_updates;       /* blocked tensor-core route: block-pair rotations applied to X (and W) */
  int32_t debug_error;      /* library built with LFA_DEBUG: the site of the first failed index
                               check (include/lfa_debug.h), 0 if none; always 0 otherwise */
} lfa_info_t;

/* Creates a plan for nlayers layers (Algorithm 1's "SVD with LFA(A, m, n)",
 * applied to a whole network). Builds the twiddle tables T_n[t] = exp(2 pi i t/n)
 * in fp64 on the host (rounded to fp32), the half-grid work list and the Jacobi
 * schedules; chooses a kernel variant per layer; allocates the plan's device
 * memory (the only allocation of the library). flags: LFA_VALUES is implied;
 * LFA_VECTORS adds U, V; LFA_HALF_OUTPUT; LFA_PLAIN. opt may be NULL.
 * On success *plan is set; on failure *plan is NULL and nothing leaks.
 * Errors: LFA_ERR_INVALID_ARG (sizes, flags, NULL plan/layers, nlayers not in
 * [1, 64]), LFA_ERR_UNSUPPORTED (no CUDA device of compute capability 10.3),
 * LFA_ERR_OOM, LFA_ERR_CUDA. */
lfa_status_t lfa_plan(lfa_plan_t* plan, const lfa_layer_desc_t* layers, int32_t nlayers,
                      uint32_t flags, const lfa_options_t* opt);

/* Forward: the SVD of every layer's operator (Sec. III, Algorithm 1).
 *  w[l]      device float32 [c_out][c_in][kh][kw]                 (input)
 *  sigma[l]  device float32 [n*m][r], or [F_h][r] with LFA_HALF_OUTPUT (output)
 *  U[l]      device complex64 [F_h][c_out][r]: U_k for the half-grid frequency k (output,
 *            required iff the plan has LFA_VECTORS, else ignored and may be NULL)
 *  V[l]      device complex64 [F_h][c_in][r]: V_k likewise.
 *            A_k = U_k diag(sigma_k) V_k^*. For the conjugate frequency -k the
 *            factors are conj(U_k), sigma_k, conj(V_k).
 * Allocates nothing; asynchronous on `stream`. Errors: LFA_ERR_INVALID_ARG
 * (NULL plan or pointer), LFA_ERR_CUDA (launch failure). */
lfa_status_t lfa_svd(lfa_plan_t plan, const float* const* w, float* const* sigma,
                     float* const* U, float* const* V, void* stream);

/* The symbols themselves (Sec. III, the c_out x c_in matrix A_k) of one layer,
 * for all half-grid frequencies: out = device complex64 [F_h][c_out][c_in].
 * Asynchronous. Errors: LFA_ERR_INVALID_ARG. */
lfa_status_t lfa_symbols(lfa_plan_t plan, int32_t layer, const float* w, float* out, void* stream);

/* The same symbols through the FFT route (plan created with LFA_FFT_ROUTE): the kernel of every
 * channel pair placed on the n x m grid at its tap offsets (aliasing taps added) and transformed
 * by cuFFT's batched real-to-complex transform, F = conj(A_k), gathered into
 * out = device complex64 [F_h][c_out][c_in]. Asynchronous. Errors: LFA_ERR_INVALID_ARG (plan
 * without LFA_FFT_ROUTE, NULL pointers), LFA_ERR_CUDA. */
lfa_status_t lfa_fft_symbols(lfa_plan_t plan, int32_t layer, const float* w, float* out, void* stream);

/* Global singular vectors (Sec. III, U^_k = F_k^out U_k, V^_k = F_k^in V_k) of one
 * layer for the flat indices q in [first, first + count), q = f*r + s over the
 * FULL grid (f = j*m + l, s = position in descending order):
 *   u_hat[q - first][o][x1][x2] = U_f[o][s] * exp(2 pi i (j x1/n + l x2/m)) / sqrt(n m)
 *   v_hat[q - first][i][x1][x2] = V_f[i][s] * exp(2 pi i (j x1/n + l x2/m)) / sqrt(n m)
 * where U_f = U[h] for a half-grid frequency f (h its position in the half grid) and
 * U_f = conj(U[h(fc)]) otherwise. U, V: the layer's lfa_svd outputs. u_hat is complex64
 * [count][c_out][n][m], v_hat complex64 [count][c_in][n][m]; either may be NULL.
 * Strided layer: v_hat is complex64 [count][c_in][s_h n][s_w m] on the fine torus, with
 *   v_hat[q - first][i][s_h x1 + u_h][s_w x2 + u_w] = V_f[(i, u)][s] exp(2 pi i (j x1/n + l x2/m)) / sqrt(n m).
 * Errors: LFA_ERR_INVALID_ARG (range outside [0, n*m*r), plan without LFA_VECTORS). */
lfa_status_t lfa_expand(lfa_plan_t plan, int32_t layer, const float* U, const float* V,
                        int64_t first, int64_t count, float* u_hat, float* v_hat, void* stream);

/* Backward: dL/dw from dL/dsigma. For a simple singular value
 * d(sigma_s) = Re(u_s^* dA_k v_s) and, from the symbol definition,
 * dA_k/dw[o,i,a,b] = exp(2 pi i <k, y_ab>) e_o e_i^T. Summed over frequencies:
 *   dw[o,i,a,b] = sum_k Re( G_k[o,i] exp(-2 pi i <k, y_ab>) ),  G_k = U_k diag(g~_k) V_k^*,
 * (strided layer: G_k[o,(i,u_ab)] and exp(-2 pi i <k, q_ab>), y_ab = s q_ab + u_ab)
 * over the half grid, with g~_k = g_k + g_{-k} for a conjugate pair and g~_k = g_k for a
 * self-conjugate k (full-grid dsigma), or g~_k = dsigma_half[k] with LFA_HALF_OUTPUT.
 * Symbols are not needed (only U, V, dsigma).
 *  dsigma[l] device float32 in sigma's layout (input)
 *  U[l], V[l] the lfa_svd outputs of the same w (input)
 *  dw[l]     device float32 [c_out][c_in][kh][kw], overwritten (output)
 * Stride-1 layers with c_out, c_in >= 128 and at most 25 taps form G_k on the tensor cores
 * (TF32 split in three, FP32 accuracy); other layers on the CUDA cores.
 * Deterministic (fixed reduction order; no float atomics). Requires a plan with
 * LFA_VECTORS (else LFA_ERR_INVALID_ARG). Allocates nothing; asynchronous (all layers in one
 * replayed CUDA graph unless the plan was created with use_graph = 0). */
lfa_status_t lfa_svd_backward(lfa_plan_t plan, const float* const* dsigma, const float* const* U,
                              const float* const* V, float* const* dw, void* stream);

/* Spectral editing modes (see lfa_spectral_edit). */
#define LFA_EDIT_CLIP       0  /* phi(s) = min(s, a): clip the spectral norm to a */
#define LFA_EDIT_CLAMP      1  /* phi(s) = min(max(s, a), b) */
#define LFA_EDIT_THRESHOLD  2  /* phi(s) = s if s >= a else 0 (hard threshold; a global low rank) */
#define LFA_EDIT_RANK       3  /* keep the first round(a) singular values of every frequency */
#define LFA_EDIT_PINV       4  /* the pseudo-inverse: phi(s) = 1/s for s > a, else 0, with the
                                  roles of U and V exchanged (a c_out -> c_in convolution) */

/* Spectral editing: the applications the paper motivates (Sec. I-II: spectral-norm
 * regularisation, low-rank compression) edit the singular values of the operator. This
 * returns, per layer, the kh x kw kernel nearest in Frobenius norm to the edited operator
 * B = U phi(S) V^* (phi applied to every singular value of every frequency):
 *   w_out[o,i,a,b] = <B, T_oiab> / (n m) = (1/(n m)) sum_k Re( B_k[o,i] exp(-2 pi i <k, y_ab>) ),
 * T_oiab the operator of one tap (these are orthogonal, <T, T> = n m, when no taps alias,
 * kh <= n and kw <= m). When the kernel covers the torus (kh = n, kw = m) the edit is exact.
 *  sigma[l], U[l], V[l]  the layer's lfa_svd outputs (plan with LFA_VECTORS)
 *  mode, a, b            LFA_EDIT_* and its parameters
 *  w_out[l]              device float32 [c_out][c_in][kh][kw], overwritten; with LFA_EDIT_PINV
 *                        [c_in][c_out][kh][kw]: the kernel of a c_out -> c_in convolution nearest
 *                        to the pseudo-inverse A^+ (symbols V_k S_k^+ U_k^*; the paper's
 *                        pseudo-inverse application, Sec. II), taps at the same offsets y_ab
 * Uses the plan's backward workspace; deterministic; asynchronous. Errors: LFA_ERR_INVALID_ARG,
 * LFA_ERR_UNSUPPORTED (LFA_EDIT_PINV on a strided layer). */
lfa_status_t lfa_spectral_edit(lfa_plan_t plan, const float* const* sigma, const float* const* U,
                               const float* const* V, int32_t mode, float a, float b,
                               float* const* w_out, void* stream);

/* dL/dsigma of the spectral regulariser L = sum_layers max(sigma) + lam * sum (sigma - 1)^2
 * (a spectral-norm term plus an orthogonality term) for each layer's sigma in the plan's
 * sigma layout: dsigma = 2 lam (sigma - 1), plus 1 at the first maximiser (row-major).
 * The max is attained at both k and -k; they are the same function of w, so one
 * representative carries the gradient. Also writes the loss value per layer to
 * loss[l] (device float32 scalar; nullable). Asynchronous. */
lfa_status_t lfa_regulariser_grad(lfa_plan_t plan, const float* const* sigma, float lam,
                                  float* const* dsigma, float* const* loss, void* stream);

/* Size in bytes of the fixed device scratch array of lfa_svd_backward_noalloc (32 MiB). */
#define LFA_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Backward pass that allocates nothing. The paper has no counterpart: it exists for
 * callers that cannot call cudaMalloc -- code whose device memory is owned entirely by
 * another allocator (a framework's caching allocator, a serving runtime that reserves
 * HBM at start-up), or a latency-critical loop that cannot pay for cudaMalloc/cudaFree,
 * which may synchronise the device. It needs no plan (lfa_plan allocates) and computes
 * what lfa_svd_backward computes for one layer:
 *   layer   host pointer to the layer description (see lfa_layer_desc_t)
 *   flags   0 (dsigma on the full grid, [n*m][r]) or LFA_HALF_OUTPUT ([F_h][r])
 *   dsigma  device float32 dL/dsigma in that layout; U, V: the layer's lfa_svd outputs
 *   dw      device float32 [c_out][c_in][kh][kw], overwritten
 * Its scratch (twiddles, half-grid list, G_k workspace, partial sums) lives in one
 * file-scope device array of LFA_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until the process exits. The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) and caches it per driver context (a
 * device reset or another current context makes the next call look it up again); make
 * that first call before any stream capture. All calls share the array and it keeps the
 * last call's contents (each call writes what it reads, nothing must start at zero);
 * calls that overlap on the GPU race. A layer needs 4*c_out*c_in*kh*kw bytes of partial
 * sums per frequency chunk. Stride-1 layers with at most 25 taps keep G_k in registers
 * and may use the whole array for partial sums (at least one chunk); other layers split
 * it: partial sums in half of it and 8*c_out*c_in*s_h*s_w bytes of G per half-grid
 * frequency of a chunk in the rest. Layers that do not fit (e.g. c_out = c_in = 512 with
 * k = 7: one chunk of partial sums is 51 MB) are rejected with LFA_ERR_UNSUPPORTED
 * before any work.
 * Asynchronous on `stream`. Errors: LFA_ERR_INVALID_ARG, LFA_ERR_UNSUPPORTED, LFA_ERR_CUDA. */
lfa_status_t lfa_svd_backward_noalloc(const lfa_layer_desc_t* layer, uint32_t flags, const float* dsigma,
                                      const float* U, const float* V, float* dw, void* stream);

/* Frees the plan's device memory and the plan. NULL is accepted. Synchronises
 * the device work the plan issued. */
lfa_status_t lfa_destroy(lfa_plan_t plan);

/* Copies the counters of the last lfa_svd into *info (synchronises the plan's
 * last stream). Returns LFA_ERR_TIMEOUT if a bounded device wait ran out, else
 * LFA_ERR_NONFINITE if a symbol had NaN/Inf, else LFA_ERR_NOT_CONVERGED if a symbol
 * hit max_sweeps, else LFA_OK. */
lfa_status_t lfa_get_info(lfa_plan_t plan, lfa_info_t* info);

/* Per-layer queries: half-grid size F_h, r, the kernel variant chosen (with
 * LFA_VARIANT_LOGGED set when the layer runs the rotation-log route), and the
 * half-grid frequency list (host int32 array of F_h entries, may be NULL). */
lfa_status_t lfa_layer_query(lfa_plan_t plan, int32_t layer, int64_t* F_h, int32_t* r,
                             int32_t* variant, int32_t* half_grid);

/* Static strings; never NULL. */
const char* lfa_status_string(lfa_status_t status);
const char* lfa_variant_name(int32_t variant);
/* The last CUDA runtime error seen by the library in this thread (cudaError_t as int). */
int32_t lfa_last_cuda_error(void);
/* Number of kernels this library has enqueued in this process so far (a replayed
 * CUDA graph counts each of its kernel nodes). Host-side counter; for launch accounting. */
int64_t lfa_kernel_launches(void);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t lfa_version(void);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif  /* LFA_H_ */
