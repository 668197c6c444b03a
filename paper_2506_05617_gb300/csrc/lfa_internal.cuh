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
  unsigned int queue[16];        // work-queue tickets, one per launch of a call
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
  int32_t item_begin;       // first work item of this layer in its launch
  float tol2;               // squared Jacobi threshold
};

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

// Auxiliary kernels (aux_kernels.cu).
cudaError_t launch_symbols(const LayerArgs& La, float2* out, cudaStream_t s);
cudaError_t launch_expand(const LayerArgs& La, const float2* U, const float2* V, int64_t first,
                          int64_t count, float2* u_hat, float2* v_hat, cudaStream_t s);
cudaError_t launch_backward(const LayerArgs& La, const float* dsigma, int half_output,
                            const float2* U, const float2* V, float2* G, int64_t g_cap,
                            float* partial, int chunks, float* dw, cudaStream_t s, int* nkernels);
cudaError_t launch_edit_values(const LayerArgs& La, int half_output, const float* sigma, int mode, float a,
                               float b, float* g, cudaStream_t s);
cudaError_t launch_regulariser(const LayerArgs& La, int half_output, const float* sigma, float lam,
                               float* dsigma, float* loss, cudaStream_t s);

}  // namespace lfa
