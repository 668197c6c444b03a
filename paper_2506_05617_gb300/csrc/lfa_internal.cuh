// Internal structures shared by the host API and the kernels of the LFA SVD
// library (arXiv 2506.05617). Not part of the public ABI (include/lfa.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lfa {

constexpr int kMaxLayers = 64;   // layers per plan
constexpr int kMaxTaps = 256;    // kh * kw <= 225 (k <= 15)

// Device counters of one lfa_svd call; reset at the start of each call.
struct Counters {
  unsigned long long unconverged;
  unsigned long long nonfinite;
  unsigned long long sweeps;
  unsigned long long rotations;
  unsigned long long timeouts;   // bounded device waits that ran out (tensor-core route)
  unsigned long long tc_grams;   // block-pair Gram matrices formed on the tensor cores
  unsigned long long tc_updates; // block-pair rotations applied on the tensor cores
  // tensor-core route, summed over CTAs (clock64 of each CTA's thread 0): Gram, inner sweep,
  // update, assembly, output, whole symbols
  unsigned long long bj_cycles[6];
  unsigned int queue[16];        // work-queue tickets, one per launch of a call
  unsigned int bw_queue[2];      // work-queue tickets of the tensor-core backward's launches
  unsigned int debug_error;      // debug build: the site id of the first failed index check
  unsigned long long warm_starts; // blocked route: symbols started from their predecessor's V
};

// One layer as a kernel sees it. The Jacobi problem of a symbol is X (M x N), with
// X = A_k (M = c_out, N = c_in) when c_out >= c_in ("tall"), else X = A_k^* (M = c_in,
// N = c_out, "wide"). N = r = min(c_out, c_in) columns are orthogonalised.
struct LayerArgs {
  const float* w;           // [c_out][c_in][kh][kw]
  float* sigma;             // full grid [n*m][r] or half grid [F_h][r]
  float2* U;                // [F_h][c_out][r]
  float2* V;                // [F_h][c_in][r]
  const int32_t* half;      // half-grid frequencies f = j*m + l, increasing, [F_h]
  const float2* tw_n;       // T_n[t] = exp(2 pi i t / n), [n]
  const float2* tw_m;       // T_m[t] = exp(2 pi i t / m), [m]
  const float2* symbols;    // materialised symbols [F_h][c_out][c_in] (plain path) or null
  int32_t c_out, c_in, kh, kw, n, m, ph, pw;
  int32_t F_h, r, M, N, wide;
  int32_t item_begin;       // first work item of this layer in its launch (blocked route: first symbol)
  // Stride (sh, sw) >= 1 and the weights' input channels c_w. The symbol has c_in = c_w sh sw
  // columns (i, u_h, u_w) -> i sh sw + u_h sw + u_w: the polyphase components of the fine input.
  int32_t c_w, sh, sw;
  float tol2;               // squared Jacobi threshold
  unsigned int* dbg;        // debug build: the word a failed index check writes its site id to
};

// Index checks of the debug build (compiled with -DLFA_DEBUG, library liblfa_debug.so): a failed
// check records its site id in the plan's debug word (the first failure wins) and the guarded
// access is skipped; the release build compiles them out. Nothing traps. Site ids are listed in
// include/lfa_debug.h.
#ifdef LFA_DEBUG
__device__ __forceinline__ bool debug_check(unsigned int* word, bool ok, unsigned int id) {
  if (!ok && word) atomicCAS(word, 0u, id);
  return ok;
}
#define LFA_DOK(word, cond, id) ::lfa::debug_check((word), (cond), (id))
#else
#define LFA_DOK(word, cond, id) true
#endif

// floor(a / s) for s >= 1: the coarse offset q of a tap y = s q + u, 0 <= u < s.
__host__ __device__ __forceinline__ int floor_div(int a, int s) { return a >= 0 ? a / s : -((s - 1 - a) / s); }

// Fills the geometry of La from a layer description (stride 0 reads as 1) after checking the
// limits that every entry point shares; false when one is violated.
inline bool set_geometry(LayerArgs& La, int c_out, int c_in, int kh, int kw, int n, int m, int pad_h,
                         int pad_w, int stride_h, int stride_w) {
  const int sh = stride_h == 0 ? 1 : stride_h, sw = stride_w == 0 ? 1 : stride_w;
  if (sh < 1 || sw < 1 || sh > 8 || sw > 8) return false;
  if (c_out < 1 || c_in < 1 || c_out > 512 || c_in > 512 || c_in * sh * sw > 512) return false;
  if (kh < 1 || kw < 1 || kh > 15 || kw > 15) return false;
  if (n < 1 || m < 1 || n > 65536 || m > 65536 || (int64_t)n * m > 0x7fffffffLL) return false;
  if (pad_h < -1 || pad_h >= kh || pad_w < -1 || pad_w >= kw) return false;
  La.c_out = c_out; La.c_w = c_in; La.sh = sh; La.sw = sw; La.c_in = c_in * sh * sw;
  La.kh = kh; La.kw = kw; La.n = n; La.m = m;
  La.ph = pad_h < 0 ? kh / 2 : pad_h;
  La.pw = pad_w < 0 ? kw / 2 : pad_w;
  La.r = c_out < La.c_in ? c_out : La.c_in;
  La.wide = La.c_in > c_out ? 1 : 0;
  La.M = c_out > La.c_in ? c_out : La.c_in;
  La.N = La.r;
  return true;
}

// exp(2 pi i <k, q_ab>) for the frequency k = (j/n, l/m) and the tap (a, b), q_ab = floor(y_ab / s)
// its coarse offset (q = y at stride 1); products below 2^31 since j < n <= 65536 and |q| < 15.
__device__ __forceinline__ float2 tap_phase(const LayerArgs& La, int j, int l, int a, int b) {
  int ia = (j * floor_div(a - La.ph, La.sh)) % La.n;
  if (ia < 0) ia += La.n;
  int ib = (l * floor_div(b - La.pw, La.sw)) % La.m;
  if (ib < 0) ib += La.m;
  const float2 p = La.tw_n[ia], q = La.tw_m[ib];
  return make_float2(p.x * q.x - p.y * q.y, p.x * q.y + p.y * q.x);
}

// Symbol entry A_k[o][i] from the taps and their phases phs[a kw + b] (symbol definition, Sec. III;
// for a stride, the taps of column i = (ci, u) are those whose offset is congruent to u).
__device__ __forceinline__ float2 symbol_entry(const LayerArgs& La, int o, int i, const float2* phs) {
  const int kk = La.kh * La.kw;
  float re = 0.f, im = 0.f;
  if (La.sh == 1 && La.sw == 1) {
    const float* wp = La.w + ((size_t)o * La.c_w + i) * kk;
    for (int t = 0; t < kk; ++t) {
      const float wv = __ldg(wp + t);
      const float2 p = phs[t];
      re = fmaf(wv, p.x, re);
      im = fmaf(wv, p.y, im);
    }
  } else {
    const int S = La.sh * La.sw;
    const int ci = i / S, u = i - ci * S, uh = u / La.sw, uw = u - uh * La.sw;
    const float* wp = La.w + ((size_t)o * La.c_w + ci) * kk;
    for (int a = (uh + La.ph) % La.sh; a < La.kh; a += La.sh)
      for (int b = (uw + La.pw) % La.sw; b < La.kw; b += La.sw) {
        const int t = a * La.kw + b;
        const float wv = __ldg(wp + t);
        const float2 p = phs[t];
        re = fmaf(wv, p.x, re);
        im = fmaf(wv, p.y, im);
      }
  }
  return make_float2(re, im);
}

// One launch of a Jacobi variant over some layers (a persistent grid pulling items).
struct JacobiLaunch {
  LayerArgs L[kMaxLayers];
  int32_t nlayers;
  int32_t total_items;
  int32_t max_sweeps;
  int32_t half_output;
  int32_t queue_slot;
  Counters* counters;
  // rotation log (symbols whose W does not fit registers): per symbol h of the launch,
  // log[(h * log_cap + t) * NP + team] = (c - 1, Re(e s), Im(e s), 0) of round t (zeros: no
  // rotation), rounds[h] = number of rounds run, xraw[h][row][column] = the final X columns in
  // column order (sigma, order and normalisation are left to the finalize kernel).
  float4* log;
  int32_t log_cap;
  int32_t* rounds;
  float2* xraw;
};

// Replay of logged rotations onto W = I (one CTA per (row block, symbol)), then the finalize
// step: sigma_c = |x_c| / |w_c|, descending order, normalised X and W columns in that order.
struct ReplayArgs {
  const float4* log;
  int32_t log_cap;
  const int32_t* rounds;
  float2* wraw;       // [symbols][N][N] W in column order
  const float2* xraw; // [symbols][M][N] X in column order
  LayerArgs La;       // the layer, half-grid list offset to the batch
  int32_t half_output;
  Counters* counters;
};
cudaError_t launch_replay(int NP, const ReplayArgs& R, int symbols, cudaStream_t s, int* nkernels);
cudaError_t prepare_replay(int NP);   // kernel attributes, once per plan
bool replay_supported(int NP);        // a replay configuration exists for NP pairs

// Blocked one-sided Jacobi on the tensor cores (blocked.cu): one CTA per symbol, X and W in a
// per-CTA workspace slot (column-major real / imaginary planes). One launch serves the layers whose
// symbols pad to the same Mp x Np; layer k's symbols are [L[k].item_begin, + L[k].F_h) of the
// launch's total_symbols.
struct BJLaunch {
  LayerArgs L[kMaxLayers];
  int32_t nlayers;
  // Warm starts (vectors; runs > 0): the launch's symbols (layer after layer, half-grid order) are
  // cut into `runs` runs of run_len consecutive symbols; item t is position p = t / runs of run
  // t % runs, symbol g = (t % runs) * run_len + p (total_items = runs * run_len, items past the
  // last symbol are skipped). done[g] != 0 once symbol g's outputs are written; the next symbol of
  // its run, in the same layer, then starts from its V, else from W = I. runs = 0: item t is
  // symbol t, every symbol starts cold.
  int32_t runs, run_len;
  int32_t total_symbols;
  int32_t* done;            // the launch's done flags (total_symbols)
  int32_t Mp, Np;           // padded rows of X (multiple of 128) and columns (multiple of 128)
  int32_t ldx, ldw;         // leading dimensions of the X and W planes
  float* ws;                // slots of slot_floats floats, one per CTA of the grid
  size_t slot_floats;
  int32_t total_items;      // work items of the launch (total_symbols without warm starts)
  int32_t max_sweeps;
  int32_t half_output;
  int32_t queue_slot;
  Counters* counters;
};
bool bj_supported(int M, int N);
int bj_min_symbols(int N);   // half-grid symbols from which the built-in choice takes the route
void bj_dims(int M, int N, int* Mp, int* Np);
size_t bj_slot_floats(int M, int N, bool vec);
cudaError_t bj_max_ctas(bool vec, int sms, int* ctas);   // co-resident CTAs (kernel attributes set)
extern int g_bj_ctas_per_sm;                             // 0: the kernel's own choice (debug hook)
extern int g_bj_max_ctas;                                // > 0: at most this many CTAs (debug hook)
extern int g_bj_runs;                                    // 0: two runs per CTA, < 0: no warm starts
cudaError_t bj_occupancy(bool vec, int* blocks, int* regs, int* smem_static, int* smem_dyn);
cudaError_t launch_bj(const BJLaunch& A, int ctas, bool vec, cudaStream_t s);
cudaError_t launch_bj_gram_test(const float* Xr, const float* Xi, int ld, int Mp, const int* cols, float* D,
                                Counters* ctr, cudaStream_t s);
cudaError_t launch_bj_update_test(const float* Pr, const float* Pi, float* Or, float* Oi, int ld, int rows,
                                  const int* cols, const float2* Q, Counters* ctr, cudaStream_t s);

// The FFT route to the symbols (fft_route.cu, cuFFT): the paper's comparison system.
int fft_chunk_pairs(const LayerArgs& La, size_t bytes);                 // channel pairs per transform batch
cudaError_t fft_make_plan(const LayerArgs& La, int pairs, void** handle);
void fft_destroy_plan(void* handle);
cudaError_t launch_fft_symbols(const LayerArgs& La, void* handle, int pairs, void* ws, float2* out, cudaStream_t s,
                               int* nk);

// Auxiliary kernels (aux_kernels.cu).
cudaError_t launch_symbols(const LayerArgs& La, float2* out, cudaStream_t s);
// chunk count of the fused backward (stride 1, at most 25 taps), or 0 when it does not apply
int fused_backward_chunks(const LayerArgs& La);
// unit vectors for the exactly zero columns of the X-side factors [symbols][M][N] of a layer
cudaError_t launch_complete(const LayerArgs& La, float2* X, int symbols, cudaStream_t s);
cudaError_t launch_expand(const LayerArgs& La, const float2* U, const float2* V, int64_t first,
                          int64_t count, float2* u_hat, float2* v_hat, cudaStream_t s);
// The backward of one layer. With `queue` (two device counters) and `ctr` given, stride-1 layers of
// 128 channels and more (tc_backward_parts > 0) take the tensor-core route (backward_tc.cu), with
// `chunks` partial slabs; otherwise the CUDA-core kernels.
cudaError_t launch_backward(const LayerArgs& La, const float* dsigma, int half_output,
                            const float2* U, const float2* V, float2* G, int64_t g_cap,
                            float* partial, int chunks, float* dw, cudaStream_t s, int* nkernels,
                            unsigned int* queue = nullptr, Counters* ctr = nullptr, int sms = 0);
// partial slabs of the tensor-core backward for a layer, 0 when the route does not apply
int tc_backward_parts(const LayerArgs& La);
cudaError_t launch_backward_tc(const LayerArgs& La, const float* dsigma, int half_output, const float2* U,
                               const float2* V, float2* G, int64_t g_cap, float* partial, int parts,
                               unsigned int* queue, Counters* ctr, float* dw, int sms, cudaStream_t s,
                               int* nkernels);
// dw = sum over `chunks` partial slabs of `total` floats, in slab order
cudaError_t launch_backward_reduce(const float* partial, int chunks, int64_t total, float* dw, cudaStream_t s);
cudaError_t launch_edit_values(const LayerArgs& La, int half_output, const float* sigma, int mode, float a,
                               float b, float* g, cudaStream_t s);
// scratch: kRegScratchBytes of device memory for the per-CTA partials (plan-owned)
constexpr size_t kRegScratchBytes = 1024;
cudaError_t launch_regulariser(const LayerArgs& La, int half_output, const float* sigma, float lam,
                               float* dsigma, float* loss, float* scratch, cudaStream_t s);

}  // namespace lfa
