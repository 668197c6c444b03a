/*
 * lfa_debug.h -- host-only hooks of the LFA SVD library that expose its plan-time
 * logic (no device work), so that it can be tested on a machine without a GPU.
 * The paper has no counterpart of these; they exist for testing the library.
 */
#ifndef LFA_DEBUG_H_
#define LFA_DEBUG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The Jacobi pair schedule for ncols (even, 2..1024) columns: one sweep of ncols-1 rounds
 * of ncols/2 pairs, as (a, b) column ids, written to out[(round*ncols/2 + team)*2 + {0,1}]
 * when out is not NULL (cap = capacity in uint16 elements). Consecutive rounds share exactly
 * one column per team, kept in the same slot; every pair occurs once per sweep.
 * Returns the number of rounds, or a negative value on invalid input (-1), a failed
 * construction (-2) or a too small buffer (-3). */
int32_t lfa_debug_schedule(int32_t ncols, uint16_t* out, int64_t cap);

/* The half-grid frequency list of an n x m torus (see lfa.h): writes it to out (cap entries)
 * when out is not NULL and returns its length F_h, or a negative value on invalid input. */
int64_t lfa_debug_half_grid(int32_t n, int32_t m, int32_t* out, int64_t cap);

/* The built-in kernel-variant choice for an M x N Jacobi problem (M = max(c_out, c_in),
 * N = min(c_out, c_in)); -1 if no register-resident variant holds it. */
int32_t lfa_debug_choose_variant(int32_t M, int32_t N, int32_t vectors);

/* Number of kernel variants (ids 0 .. count-1, named by lfa_variant_name). */
int32_t lfa_debug_variant_count(void);

/* The route an autotuner cache file (text lines "M N vectors variant [log]") selects for an
 * M x N problem: the variant id, with LFA_VARIANT_LOGGED set for the rotation-log route; -1 when
 * the file has no usable line for it (missing, or a variant that cannot hold the problem). */
int32_t lfa_debug_tuned_variant(const char* path, int32_t M, int32_t N, int32_t vectors);

/* Position in the half-grid list of the representative of full-grid frequency f (f itself or
 * its conjugate), the closed form the lifting kernel uses; -1 on invalid input. */
int64_t lfa_debug_half_position(int32_t n, int32_t m, int32_t f);

/* 1 if variant v holds an M x N problem in registers (with the accumulated rotations W when
 * vectors != 0, which needs a variant built with vectors), else 0: the rule the built-in choice
 * and the autotuner cache apply. */
int32_t lfa_debug_variant_fits(int32_t v, int32_t M, int32_t N, int32_t vectors);

/* 1 if values variant v can serve vectors through the rotation log and the W replay for an
 * M x N problem (a replay configuration exists for its pairs), else 0. */
int32_t lfa_debug_logged_ok(int32_t v, int32_t M, int32_t N);

/* The contiguous half-grid range [*first, *first + *count) that shard `rank` of `count_shards`
 * decomposes for an n x m torus (lfa_options_t.shard_rank / shard_count): [floor(r F_h / R),
 * floor((r + 1) F_h / R)). Returns F_h, or -1 on invalid input. */
int64_t lfa_debug_shard_range(int32_t n, int32_t m, int32_t rank, int32_t count_shards, int64_t* first,
                              int64_t* count);

/* The two tensor-core contractions of the blocked Jacobi route (tcgen05, TF32 operands split into
 * hi + lo, three products, FP32 accumulation), run by one CTA on caller data; they let tests check
 * the MMA operand layouts and the 3xTF32 accuracy apart from the Jacobi iteration.
 * lfa_debug_tc_gram: H = Y^* Y (complex64 [64][64] to D) for Y = the 64 columns cols[] (device
 *   int32) of the column-major planes (Xr, Xi) (leading dimension ld, a multiple of 4, >= Mp),
 *   rows [0, Mp), Mp a multiple of 32.
 * lfa_debug_tc_update: (Or, Oi)[cols] = Y Q over rows [0, rows) (a multiple of 128), Y the columns
 *   cols[] of (Pr, Pi), Q device complex64 [64][64] row-major.
 * Both return 0, -1 on invalid arguments, or a CUDA error code; asynchronous on `stream`. */
int32_t lfa_debug_tc_gram(const float* Xr, const float* Xi, int32_t ld, int32_t Mp, const int32_t* cols, float* D,
                          void* stream);
int32_t lfa_debug_tc_update(const float* Pr, const float* Pi, float* Or, float* Oi, int32_t ld, int32_t rows,
                            const int32_t* cols, const float* Q, void* stream);

/* The backward route a layer takes in lfa_svd_backward: 2 the tensor-core G product (stride 1,
 * c_out and c_in >= 128, at most 25 taps), 1 the fused CUDA-core kernel (stride 1, at most 25 taps),
 * 0 the CUDA-core G product and tap projection; -1 for an invalid layer. */
int32_t lfa_debug_backward_route(int32_t c_out, int32_t c_in, int32_t kh, int32_t kw, int32_t stride_h,
                                 int32_t stride_w);

/* Phase profile of the blocked tensor-core route in the last lfa_svd call of a plan (waits for the
 * plan's last stream): out[0..5] = clock cycles summed over the route's CTAs (thread 0 of each) in
 * block-pair Grams, inner sweeps, updates, symbol assembly (with a warm start's product), output,
 * and whole symbols; out[6] = symbols that started warm (from the V of the previous symbol of their
 * run); *ctas = the CTAs of the route's launch for the plan's first blocked layer (0 when no layer
 * takes the route). out holds 7 entries. plan is an lfa_plan_t. Returns an lfa_status_t (0 on
 * success, 1 on a NULL argument). */
int32_t lfa_debug_bj_profile(void* plan, uint64_t* out, int32_t* ctas);
/* Co-resident CTAs per SM of the blocked route in plans created afterwards: 0 restores the
 * kernel's own choice (two), 1 launches one per SM. For launch-shape measurements. */
void lfa_debug_set_bj_ctas_per_sm(int32_t n);
/* Launch shape of the blocked route in plans created afterwards: at most max_ctas CTAs (<= 0: the
 * kernel's own count), and `runs` runs of neighbouring symbols per layer for the warm starts with
 * vectors (0: two per CTA, the default; < 0: no warm starts, every symbol starts from W = I). For
 * tests of the warm starts on small layers and for measurements. */
void lfa_debug_set_bj_grid(int32_t max_ctas, int32_t runs);
/* Resources of the blocked route's kernel (values-only or with vectors): out[0] = CTAs per SM the
 * occupancy calculator admits, out[1] = registers per thread, out[2] = static and out[3] = dynamic
 * shared memory per CTA in bytes, out[4] = CTAs per SM with 32 KB of dynamic shared memory instead.
 * Returns an lfa_status_t. */
int32_t lfa_debug_bj_occupancy(int32_t vectors, int32_t* out);

/* Site ids of the index checks of the debug build (liblfa_debug.so, built with -DLFA_DEBUG; the
 * release library has none): lfa_info_t.debug_error holds the first failed one, and lfa_get_info
 * then returns LFA_ERR_CUDA. The guarded access is skipped, never trapped.
 *   1  element-wise Jacobi, cluster variants: output rank of a column, or symbol index
 *   2  element-wise Jacobi, single-CTA variants: output rank of a column (staging mailbox)
 *   4  rotation-log finalize: output rank or symbol index
 *   5  blocked route: work item -> (layer, symbol)
 *   6  blocked route: output rank of a column
 *   7  lifting: half-grid position of a frequency
 *   8  CUDA-core backward G: symbol index
 *   9  tensor-core backward G: work item -> symbol
 *   10 tensor-core backward tap projection: part or frequency range */

#ifdef __cplusplus
}
#endif

#endif /* LFA_DEBUG_H_ */
