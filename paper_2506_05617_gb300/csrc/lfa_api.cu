// Host implementation of the C ABI declared in include/lfa.h (LFA SVD of periodic
// convolutions, arXiv 2506.05617). Plans own tables, counters and workspace; all
// per-call buffers belong to the caller.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <memory>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "../../include/lfa.h"
#include "../../include/lfa_debug.h"
#include "half_grid.cuh"
#include "jacobi_variants.cuh"
#include "lfa_internal.cuh"

using namespace lfa;

namespace {

// NVTX range around an entry point (shows the host side of each call on a profiler timeline; a no-op
// unless a profiler has injected its NVTX library).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

thread_local int32_t g_last_cuda_error = 0;
std::atomic<int64_t> g_launches{0};

lfa_status_t from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LFA_OK;
  g_last_cuda_error = (int32_t)e;
  if (e == cudaErrorMemoryAllocation) return LFA_ERR_OOM;
  return LFA_ERR_CUDA;
}

#define LFA_CUDA_TRY(expr)                          \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return from_cuda(_e);    \
  } while (0)

// Host fault injection for failure-detection tests: LFA_FAULT_INJECT=alloc|launch|nonconverge.
bool fault(const char* what) {
  const char* v = std::getenv("LFA_FAULT_INJECT");
  return v != nullptr && std::strstr(v, what) != nullptr;
}

// --------------------------------------------------------------------------- half grid
// Frequencies f = j*m + l with f <= fc, fc the index of -k; increasing order.
// Half-grid range [first, first + count) of shard r of R: [floor(r F_h / R), floor((r + 1) F_h / R)).
void shard_range(int64_t F_h, int r, int R, int64_t* first, int64_t* count) {
  const int64_t a = F_h * r / R, b = F_h * (r + 1) / R;
  *first = a;
  *count = b - a;
}

void build_half_grid(int n, int m, std::vector<int32_t>& out) {
  out.clear();
  for (int j = 0; j < n; ++j)
    for (int l = 0; l < m; ++l) {
      const int f = j * m + l;
      const int fc = ((n - j) % n) * m + (m - l) % m;
      if (f <= fc) out.push_back(f);
    }
}

// --------------------------------------------------------------------------- schedule
// The Jacobi pair schedule the kernel follows, written out on the host (for tests): the
// circle-method round robin over NC columns, team k at position k on even rounds and at
// pi(k) on odd ones, pi = (1 2)(3 4)...(NP-3 NP-2). Position i holds (c(t+i), c(t-i)),
// position 0 holds (c(t), NC-1), c(x) = x mod NC-1. Returns false for odd NC.
bool build_schedule(int NC, std::vector<ushort2>& out) {
  if (NC < 2 || (NC & 1)) return false;
  const int NP = NC / 2, Cn = NC - 1;
  auto pi = [&](int p) { return (p == 0 || p == NP - 1) ? p : ((p & 1) ? p + 1 : p - 1); };
  out.assign((size_t)Cn * NP, ushort2{0, 0});
  for (int t = 0; t < Cn; ++t)
    for (int k = 0; k < NP; ++k) {
      const int i = (t & 1) ? pi(k) : k;
      const int a = (t + i) % Cn;
      const int b = i == 0 ? NC - 1 : ((t - i) % Cn + Cn) % Cn;
      out[(size_t)t * NP + k] = ushort2{(unsigned short)a, (unsigned short)b};
    }
  std::vector<char> hit((size_t)NC * NC, 0);
  for (int t = 0; t < Cn; ++t)
    for (int k = 0; k < NP; ++k) {
      const int a = out[(size_t)t * NP + k].x, b = out[(size_t)t * NP + k].y;
      if (a == b) return false;
      const size_t idx = (size_t)std::min(a, b) * NC + std::max(a, b);
      if (hit[idx]) return false;
      hit[idx] = 1;
    }
  return true;
}

// --------------------------------------------------------------------------- variants
struct VDesc { int NP, L, MR, WR, CS, vec_ok, PPT; };
const VDesc kVariants[] = {
#define LFA_VD(id, NP, L, MR, WR, CS, OK, MB, PPT) {NP, L, MR, WR, CS, OK, PPT},
    LFA_JACOBI_VARIANTS(LFA_VD)
#undef LFA_VD
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
const char* kVariantNames[] = {
#define LFA_VN(id, NP, L, MR, WR, CS, OK, MB, PPT) \
  "reg_np" #NP "_l" #L "_mr" #MR "_wr" #WR "_cs" #CS "_ppt" #PPT,
    LFA_JACOBI_VARIANTS(LFA_VN)
#undef LFA_VN
};

int variant_rows(int v) { return kVariants[v].MR * kVariants[v].L; }
int variant_cols(int v, bool vec) {
  const int c = 2 * kVariants[v].NP;
  return vec ? std::min(c, kVariants[v].WR * kVariants[v].L) : c;
}
bool variant_fits(int v, int M, int N, bool vec) {
  return v >= 0 && v < kNumVariants && (!vec || kVariants[v].vec_ok) && M <= variant_rows(v) &&
         N <= variant_cols(v, vec);
}
// Default choice: the smallest padded problem (2*NP columns x MR*L rows) that holds M x N;
// ties go to the smaller cluster, then to one team per thread (the rotation log needs it),
// then to fewer threads per symbol (fewer butterfly levels and a cheaper barrier per round).
// An autotuner cache overrides this per problem.
int choose_variant(int M, int N, bool vec) {
  int best = -1;
  long best_area = 0;
  for (int v = 0; v < kNumVariants; ++v) {
    if (!variant_fits(v, M, N, vec)) continue;
    const long area = (long)(2 * kVariants[v].NP) * variant_rows(v);
    bool better = best < 0 || area < best_area;
    if (!better && area == best_area) {
      const VDesc& a = kVariants[v];
      const VDesc& b = kVariants[best];
      better = a.CS < b.CS || (a.CS == b.CS && a.PPT < b.PPT) ||
               (a.CS == b.CS && a.PPT == b.PPT && a.NP * a.L < b.NP * b.L);
    }
    if (better) {
      best = v;
      best_area = area;
    }
  }
  return best;
}

cudaError_t vprepare(int id, bool vec, bool fused) {
  if (vec && fused) return jacobi_vec_fused_prepare(id);
  if (!vec && fused) return jacobi_val_fused_prepare(id);
  if (!vec && !fused) return jacobi_val_plain_prepare(id);
  return cudaErrorInvalidValue;
}
cudaError_t vgrid(int id, bool vec, bool fused, int sms, int* g) {
  if (vec && fused) return jacobi_vec_fused_grid(id, sms, g);
  if (!vec && fused) return jacobi_val_fused_grid(id, sms, g);
  if (!vec && !fused) return jacobi_val_plain_grid(id, sms, g);
  return cudaErrorInvalidValue;
}
cudaError_t vlaunch(int id, bool vec, bool fused, const JacobiLaunch& P, int grid, cudaStream_t s) {
  if (vec && fused) return jacobi_vec_fused_launch(id, P, grid, s);
  if (!vec && fused) return jacobi_val_fused_launch(id, P, grid, s);
  if (!vec && !fused) return jacobi_val_plain_launch(id, P, grid, s);
  return cudaErrorInvalidValue;
}
int variant_spu(int id) {
  const int TC = kVariants[id].NP / kVariants[id].CS / kVariants[id].PPT * kVariants[id].L;
  return TC <= 32 ? 32 / TC : 1;
}
int variant_cs(int id) { return kVariants[id].CS; }

// The rotation-log route for vectors: values-mode variant v logs its rotations, W is replayed.
bool logged_ok(int v, int M, int N) {
  return variant_fits(v, M, N, false) && kVariants[v].PPT == 1 && replay_supported(kVariants[v].NP) &&
         kVariants[v].NP * kVariants[v].L / kVariants[v].CS >= 32 && N <= 512;
}

// Optional autotuner cache: text lines "M N vec variant [log|blocked]" (first match wins); "log"
// marks the rotation-log route (returned as variant | LFA_VARIANT_LOGGED), "blocked" the blocked
// tensor-core route (returned as LFA_VARIANT_BLOCKED).
int tuned_variant(const char* path, int M, int N, bool vec) {
  if (path == nullptr || path[0] == 0) return -1;
  FILE* fh = std::fopen(path, "r");
  if (!fh) return -1;
  int m, n, v, id, found = -1;
  char line[256], word[16];
  bool log = false, blk = false;
  while (std::fgets(line, sizeof line, fh)) {
    if (line[0] == '#') continue;
    word[0] = 0;
    const int got = std::sscanf(line, "%d %d %d %d %15s", &m, &n, &v, &id, word);
    if (got >= 4 && m == M && n == N && (v != 0) == vec) {
      found = id;
      log = got == 5 && std::strcmp(word, "log") == 0;
      blk = got == 5 && std::strcmp(word, "blocked") == 0;
      break;
    }
  }
  std::fclose(fh);
  if (log) return vec && logged_ok(found, M, N) ? (found | LFA_VARIANT_LOGGED) : -1;
  if (blk || found == LFA_VARIANT_BLOCKED) return bj_supported(M, N) ? LFA_VARIANT_BLOCKED : -1;
  return variant_fits(found, M, N, vec) ? found : -1;
}

}  // namespace

// ============================================================================= plan
struct lfa_plan_s {
  int nlayers = 0;
  uint32_t flags = 0;
  bool vec = false, half_output = false, plain = false, use_graph = true, fft = false, reproducible = false;
  int max_sweeps = 30;
  float tol_opt = 0.f;
  int device = 0, sms = 0;
  std::vector<lfa_layer_desc_t> desc;
  std::vector<LayerArgs> args;        // device table pointers filled, per-call pointers not
  std::vector<int> variant;           // per layer
  std::vector<std::vector<int32_t>> half_host;   // the plan's (shard of the) half grid per layer
  int shard_rank = 0, shard_count = 1;
  std::vector<int64_t> shard_first;               // position of the shard's first frequency in the half grid
  // variant groups: one persistent launch each
  struct Group { int variant; std::vector<int> layers; int items; int grid; };
  std::vector<Group> groups;
  std::vector<int> plain_grid;            // per layer (plain path)
  // layers whose W does not fit registers: values-mode forward with a rotation log + replay
  struct Logged { int layer; int variant; int grid; int batch; int log_cap; int sweeps_cap; };
  std::vector<Logged> logged;
  // layers on the blocked tensor-core route, and their launches: one persistent launch per group of
  // layers whose symbols pad to the same Mp x Np (indices into `blocked`), with its CTA count
  struct Blocked { int layer; int ctas; int sym_begin; };   // sym_begin: the layer's first done flag
  std::vector<Blocked> blocked;
  struct BlockedGroup { std::vector<int> members; int ctas; int Mp, Np; int runs; };
  std::vector<BlockedGroup> bj_groups;
  float* bj_ws = nullptr;
  int32_t* bj_done = nullptr;   // done flags of the blocked layers' symbols (warm starts)
  int bj_symbols = 0;
  float4* log_ws = nullptr;
  int32_t* rounds_ws = nullptr;
  float2* xraw_ws = nullptr;
  float2* wraw_ws = nullptr;
  // device memory
  void* dmem = nullptr;
  size_t dbytes = 0;
  Counters* counters = nullptr;
  float2* sym_ws = nullptr;  // plain path symbols [F_h][c_out][c_in] (largest layer)
  float2* g_ws = nullptr;    // backward G workspace
  int64_t g_cap_bytes = 0;
  float* partial_ws = nullptr;
  float* edit_ws = nullptr;                 // phi(sigma) / (n m) of one layer (spectral editing)
  float* reg_ws = nullptr;                  // per-CTA partials of the regulariser
  std::vector<int> bw_chunks;      // per layer
  // FFT route: a batched cuFFT plan per layer and one workspace for the real grids and spectra
  std::vector<void*> fft_plans;
  std::vector<int> fft_pairs;
  void* fft_ws = nullptr;
  // independent parts of a forward (each element-wise group; all blocked groups; all logged
  // batches) run on their own streams, forked from and joined back into the caller's stream (under
  // capture: parallel branches of the graph)
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  // graph cache
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> graph_key;
  // the backward of all layers, captured once per set of buffers like the forward
  cudaGraph_t bw_graph = nullptr;
  cudaGraphExec_t bw_exec = nullptr;
  std::vector<const void*> bw_key;
  int64_t bw_kernels = 0;                 // kernels in the captured backward
  cudaStream_t last_stream = nullptr;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool layer_geometry(const lfa_layer_desc_t& d, LayerArgs& La) {
  return set_geometry(La, d.c_out, d.c_in, d.kh, d.kw, d.n, d.m, d.pad_h, d.pad_w, d.stride_h, d.stride_w);
}

lfa_status_t validate_layer(const lfa_layer_desc_t& d) {
  LayerArgs La;
  return layer_geometry(d, La) ? LFA_OK : LFA_ERR_INVALID_ARG;
}

// Default Jacobi threshold. One-sided Jacobi on X keeps X w_p = x_p to rounding, so for a tall
// symbol (X = A_k) A v = sigma u holds exactly and the threshold only has to stay above the fp32
// noise of the M-term dot products: max(2^-22, 4 sqrt(M) 2^-24). A wide symbol is decomposed as
// X = A_k^*, and there A v - sigma u = W (X^* x_p - sigma_p^2 e_p) / sigma_p is bounded by the final
// column orthogonality, tau ||A_k||_F: its threshold is capped at 2^-20 (~9.5e-7), which keeps
// that residual below 1e-5 sigma_max for 512-column symbols at ~1 more sweep.
float default_tol(int M, bool wide) {
  const float t = std::max(4.f * std::sqrt((float)M) * std::ldexp(1.f, -24), std::ldexp(1.f, -22));
  return wide ? std::min(t, std::ldexp(1.f, -20)) : t;
}

void free_plan(lfa_plan_s* p) {
  if (!p) return;
  for (void* h : p->fft_plans)
    if (h) fft_destroy_plan(h);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->bw_exec) cudaGraphExecDestroy(p->bw_exec);
  if (p->bw_graph) cudaGraphDestroy(p->bw_graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  for (cudaStream_t b : p->branch)
    if (b) cudaStreamDestroy(b);
  for (cudaEvent_t e : p->join)
    if (e) cudaEventDestroy(e);
  if (p->fork) cudaEventDestroy(p->fork);
  if (p->dmem) cudaFree(p->dmem);
  delete p;
}

// One element-wise variant group of a forward: one persistent launch over all its layers (queue slot
// gi), then the completion of zero columns for cluster variants with vectors.
lfa_status_t enqueue_group(lfa_plan_s* p, int gi, const float* const* w, float* const* sigma, float* const* U,
                           float* const* V, cudaStream_t s) {
  const auto& g = p->groups[gi];
  {
    JacobiLaunch P{};
    int items = 0;
    for (size_t k = 0; k < g.layers.size(); ++k) {
      const int l = g.layers[k];
      LayerArgs La = p->args[l];
      La.w = w[l];
      La.sigma = sigma[l];
      La.U = p->vec ? reinterpret_cast<float2*>(U[l]) : nullptr;
      La.V = p->vec ? reinterpret_cast<float2*>(V[l]) : nullptr;
      La.item_begin = items;
      P.L[k] = La;
      items += (La.F_h + variant_spu(g.variant) - 1) / variant_spu(g.variant);
    }
    P.nlayers = (int)g.layers.size();
    P.total_items = items;
    P.max_sweeps = p->max_sweeps;
    P.half_output = p->half_output;
    P.queue_slot = gi;
    P.counters = p->counters;
    LFA_CUDA_TRY(vlaunch(g.variant, p->vec, true, P, g.grid, s));
    // cluster variants write zero vectors for negligible singular values: complete them
    if (p->vec && kVariants[g.variant].CS > 1)
      for (int k = 0; k < P.nlayers; ++k)
        LFA_CUDA_TRY(launch_complete(P.L[k], P.L[k].wide ? P.L[k].V : P.L[k].U, P.L[k].F_h, s));
  }
  return LFA_OK;
}

lfa_status_t enqueue_blocked(lfa_plan_s* p, const float* const* w, float* const* sigma, float* const* U,
                             float* const* V, cudaStream_t s) {
  // blocked layers: one persistent launch per group of same-size layers (queue slot 14), then the
  // completion of zero columns per layer
  if (p->bj_done)
    LFA_CUDA_TRY(cudaMemsetAsync(p->bj_done, 0, (size_t)p->bj_symbols * sizeof(int32_t), s));
  for (const auto& bg : p->bj_groups) {
    // BJLaunch holds kMaxLayers layers (~10 KB): built on the heap, passed by value at launch
    std::unique_ptr<BJLaunch> A(new (std::nothrow) BJLaunch());
    if (!A) return LFA_ERR_OOM;
    int items = 0;
    for (size_t k = 0; k < bg.members.size(); ++k) {
      const int l = p->blocked[bg.members[k]].layer;
      LayerArgs& La = A->L[k];
      La = p->args[l];
      La.w = w[l];
      La.sigma = sigma[l];
      La.U = p->vec ? reinterpret_cast<float2*>(U[l]) : nullptr;
      La.V = p->vec ? reinterpret_cast<float2*>(V[l]) : nullptr;
      La.item_begin = items;   // the layer's first symbol in the launch
      items += La.F_h;
    }
    A->nlayers = (int)bg.members.size();
    A->total_symbols = items;
    A->runs = bg.runs;
    A->run_len = bg.runs > 0 ? (items + bg.runs - 1) / bg.runs : 1;
    // the group's layers have consecutive done flags
    A->done = p->bj_done ? p->bj_done + p->blocked[bg.members[0]].sym_begin : nullptr;
    if (bg.runs > 0) items = bg.runs * A->run_len;
    A->Mp = bg.Mp;
    A->Np = bg.Np;
    A->ldx = bg.Mp;
    A->ldw = bg.Np;
    A->ws = p->bj_ws;
    A->slot_floats = bj_slot_floats(bg.Mp, bg.Np, p->vec);
    A->total_items = items;
    A->max_sweeps = p->max_sweeps;
    A->half_output = p->half_output;
    A->queue_slot = 14;
    A->counters = p->counters;
    LFA_CUDA_TRY(cudaMemsetAsync(&p->counters->queue[14], 0, sizeof(unsigned), s));
    LFA_CUDA_TRY(launch_bj(*A, bg.ctas, p->vec, s));
    if (p->vec)
      for (int k = 0; k < A->nlayers; ++k)
        LFA_CUDA_TRY(launch_complete(A->L[k], A->L[k].wide ? A->L[k].V : A->L[k].U, A->L[k].F_h, s));
  }
  return LFA_OK;
}

lfa_status_t enqueue_logged(lfa_plan_s* p, const float* const* w, float* const* sigma, float* const* U,
                            float* const* V, cudaStream_t s) {
  // logged layers: per batch of symbols, the values-mode forward that logs its rotations and
  // writes sigma and the X-side vectors, then the replay that builds W
  for (const auto& lg : p->logged) {
    const LayerArgs& base = p->args[lg.layer];
    const int NP = kVariants[lg.variant].NP;
    for (int b0 = 0; b0 < base.F_h; b0 += lg.batch) {
      const int cnt = std::min(lg.batch, base.F_h - b0);
      LayerArgs La = base;
      La.w = w[lg.layer];
      La.half = base.half + b0;
      La.F_h = cnt;
      La.item_begin = 0;
      La.sigma = sigma[lg.layer] + (p->half_output ? (size_t)b0 * base.r : 0);
      La.U = reinterpret_cast<float2*>(U[lg.layer]) + (size_t)b0 * base.c_out * base.r;
      La.V = reinterpret_cast<float2*>(V[lg.layer]) + (size_t)b0 * base.c_in * base.r;
      JacobiLaunch P{};
      P.L[0] = La;
      P.nlayers = 1;
      P.total_items = cnt;
      P.max_sweeps = lg.sweeps_cap;
      P.half_output = p->half_output;
      P.queue_slot = 15;
      P.counters = p->counters;
      P.log = p->log_ws;
      P.log_cap = lg.log_cap;
      P.rounds = p->rounds_ws;
      P.xraw = p->xraw_ws;
      LFA_CUDA_TRY(cudaMemsetAsync(&p->counters->queue[15], 0, sizeof(unsigned), s));
      const int cs = kVariants[lg.variant].CS;
      const int grid = std::max(cs, std::min(cnt * cs, lg.grid) / cs * cs);
      LFA_CUDA_TRY(jacobi_val_log_launch(lg.variant, P, grid, s));
      ReplayArgs R;
      R.log = p->log_ws;
      R.log_cap = lg.log_cap;
      R.rounds = p->rounds_ws;
      R.wraw = p->wraw_ws;
      R.xraw = p->xraw_ws;
      R.La = La;
      R.half_output = p->half_output;
      R.counters = p->counters;
      int nk = 0;
      LFA_CUDA_TRY(launch_replay(NP, R, cnt, s, &nk));
      LFA_CUDA_TRY(launch_complete(La, La.wide ? La.V : La.U, cnt, s));
    }
  }
  return LFA_OK;
}

// Enqueue the forward work of one call on stream s (used directly or under capture).
lfa_status_t enqueue_forward(lfa_plan_s* p, const float* const* w, float* const* sigma,
                             float* const* U, float* const* V, cudaStream_t s) {
  LFA_CUDA_TRY(cudaMemsetAsync(p->counters, 0, sizeof(Counters), s));
  if (fault("launch")) return from_cuda(cudaErrorLaunchFailure);
  if (p->plain) {
    // plain per-layer path: materialise the symbols, then one Jacobi launch per layer
    for (int l = 0; l < p->nlayers; ++l) {
      LayerArgs La = p->args[l];
      La.w = w[l];
      La.sigma = sigma[l];
      La.symbols = p->sym_ws;
      La.item_begin = 0;
      if (p->fft) {
        int nk = 0;
        LFA_CUDA_TRY(launch_fft_symbols(La, p->fft_plans[l], p->fft_pairs[l], p->fft_ws, p->sym_ws, s, &nk));
        g_launches += nk;
      } else {
        LFA_CUDA_TRY(launch_symbols(La, p->sym_ws, s));
        g_launches += 1;
      }
      JacobiLaunch P{};
      P.L[0] = La;
      P.nlayers = 1;
      const int spu = variant_spu(p->variant[l]);
      P.total_items = (La.F_h + spu - 1) / spu;
      P.max_sweeps = p->max_sweeps;
      P.half_output = p->half_output;
      P.queue_slot = l % 16;
      P.counters = p->counters;
      const int grid = p->plain_grid[l];
      if (l >= 16) LFA_CUDA_TRY(cudaMemsetAsync(&p->counters->queue[l % 16], 0, sizeof(unsigned), s));
      LFA_CUDA_TRY(vlaunch(p->variant[l], false, false, P, grid, s));
      g_launches += 1;
    }
    return LFA_OK;
  }
  // the parts of the forward, each a function of the stream it is enqueued on
  std::vector<std::function<lfa_status_t(cudaStream_t)>> parts;
  for (size_t gi = 0; gi < p->groups.size(); ++gi)
    parts.push_back([=](cudaStream_t st) { return enqueue_group(p, (int)gi, w, sigma, U, V, st); });
  if (!p->bj_groups.empty())
    parts.push_back([=](cudaStream_t st) { return enqueue_blocked(p, w, sigma, U, V, st); });
  if (!p->logged.empty())
    parts.push_back([=](cudaStream_t st) { return enqueue_logged(p, w, sigma, U, V, st); });
  if (parts.size() <= 1 || p->branch.size() < parts.size()) {
    for (auto& f : parts) {
      const lfa_status_t st = f(s);
      if (st != LFA_OK) return st;
    }
    return LFA_OK;
  }
  LFA_CUDA_TRY(cudaEventRecord(p->fork, s));
  for (size_t k = 0; k < parts.size(); ++k) {
    LFA_CUDA_TRY(cudaStreamWaitEvent(p->branch[k], p->fork, 0));
    const lfa_status_t st = parts[k](p->branch[k]);
    if (st != LFA_OK) return st;
    LFA_CUDA_TRY(cudaEventRecord(p->join[k], p->branch[k]));
    LFA_CUDA_TRY(cudaStreamWaitEvent(s, p->join[k], 0));
  }
  return LFA_OK;
}

// Kernels of one forward beyond one per group: per logged batch the logging forward, the
// replay, the finalize and the completion; per layer of a cluster group with vectors, the
// completion (one launch per 65535 symbols).
int64_t logged_launches(const lfa_plan_s* p) {
  int64_t n = 0;
  for (const auto& lg : p->logged) {
    const int batches = (p->args[lg.layer].F_h + lg.batch - 1) / lg.batch;
    n += 4 * (int64_t)batches;
  }
  if (p->vec)
    for (const auto& g : p->groups)
      if (kVariants[g.variant].CS > 1)
        for (int l : g.layers) n += (p->args[l].F_h + 65534) / 65535;
  n += (int64_t)p->bj_groups.size();
  for (const auto& bl : p->blocked) n += p->vec ? (p->args[bl.layer].F_h + 65534) / 65535 : 0;
  return n;
}

}  // namespace

extern "C" {

lfa_status_t lfa_plan(lfa_plan_t* plan, const lfa_layer_desc_t* layers, int32_t nlayers,
                      uint32_t flags, const lfa_options_t* opt) {
  NvtxRange nvtx_range("lfa_plan");
  if (plan == nullptr) return LFA_ERR_INVALID_ARG;
  *plan = nullptr;
  if (layers == nullptr || nlayers < 1 || nlayers > kMaxLayers) return LFA_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)(LFA_VALUES | LFA_VECTORS | LFA_HALF_OUTPUT | LFA_PLAIN | LFA_FFT_ROUTE | LFA_REPRODUCIBLE))
    return LFA_ERR_INVALID_ARG;
  if (flags & LFA_FFT_ROUTE) {
    flags |= LFA_PLAIN;
    for (int l = 0; l < nlayers; ++l)
      if ((layers[l].stride_h > 1) || (layers[l].stride_w > 1)) return LFA_ERR_UNSUPPORTED;
  }
  if ((flags & LFA_PLAIN) && (flags & LFA_VECTORS)) return LFA_ERR_INVALID_ARG;  // plain = values only
  for (int l = 0; l < nlayers; ++l) {
    lfa_status_t st = validate_layer(layers[l]);
    if (st != LFA_OK) return st;
  }
  if (opt && (opt->max_sweeps > 1000 || !(opt->tol < 1.f))) return LFA_ERR_INVALID_ARG;
  const int shard_count = (opt && opt->shard_count > 1) ? opt->shard_count : 1;
  const int shard_rank = opt ? opt->shard_rank : 0;
  if (shard_count > 65536 || shard_rank < 0 || shard_rank >= shard_count) return LFA_ERR_INVALID_ARG;
  if (fault("alloc")) return LFA_ERR_OOM;

  int dev = 0;
  LFA_CUDA_TRY(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  LFA_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  if (prop.major != 10 || prop.minor != 3) return LFA_ERR_UNSUPPORTED;

  lfa_plan_s* p = new (std::nothrow) lfa_plan_s();
  if (!p) return LFA_ERR_OOM;
  p->nlayers = nlayers;
  p->flags = flags;
  p->vec = (flags & LFA_VECTORS) != 0;
  p->half_output = (flags & LFA_HALF_OUTPUT) != 0;
  p->plain = (flags & LFA_PLAIN) != 0;
  p->fft = (flags & LFA_FFT_ROUTE) != 0;
  p->reproducible = (flags & LFA_REPRODUCIBLE) != 0;
  p->max_sweeps = (opt && opt->max_sweeps > 0) ? opt->max_sweeps : 30;
  if (fault("nonconverge")) p->max_sweeps = 1;
  p->tol_opt = opt ? opt->tol : 0.f;
  p->use_graph = !(opt && opt->use_graph == 0) && !p->plain;
  p->device = dev;
  p->sms = prop.multiProcessorCount;
  p->desc.assign(layers, layers + nlayers);
  p->args.resize(nlayers);
  p->variant.resize(nlayers);
  p->half_host.resize(nlayers);
  p->bw_chunks.resize(nlayers);
  p->plain_grid.assign(nlayers, 1);
  p->shard_rank = shard_rank;
  p->shard_count = shard_count;
  p->shard_first.assign(nlayers, 0);

  // ---- per-layer host tables and variant choice
  size_t bytes = align256(sizeof(Counters));
  std::vector<size_t> off_half(nlayers), off_twn(nlayers), off_twm(nlayers);
  size_t sym_bytes = 0, g_need = 0, part_bytes = 0, log_bytes = 0, ranks_bytes = 0, rounds_bytes = 0;
  size_t wraw_bytes = 0, bj_bytes = 0;
  for (int l = 0; l < nlayers; ++l) {
    const lfa_layer_desc_t& d = layers[l];
    LayerArgs& La = p->args[l];
    std::memset(&La, 0, sizeof La);
    layer_geometry(d, La);   // validated above
    build_half_grid(d.n, d.m, p->half_host[l]);
    if (shard_count > 1) {
      int64_t first = 0, count = 0;
      shard_range((int64_t)p->half_host[l].size(), shard_rank, shard_count, &first, &count);
      std::vector<int32_t> part(p->half_host[l].begin() + first, p->half_host[l].begin() + first + count);
      p->half_host[l].swap(part);
      p->shard_first[l] = first;
    }
    La.F_h = (int)p->half_host[l].size();
    const float tol = p->tol_opt > 0.f ? p->tol_opt : default_tol(La.M, La.wide != 0);
    La.tol2 = tol * tol;
    int v = -1;
    bool logged = false;
    const bool can_log = p->vec && !p->plain;
    // a requested (option, then autotuner cache) variant, possibly with the rotation-log route
    const int requested[2] = {opt ? opt->variant : -1, tuned_variant(opt ? opt->tune_cache : nullptr, La.M, La.N, p->vec)};
    bool blocked = false;
    for (int q = 0; q < 2; ++q) {
      const int rq = requested[q];
      if (v >= 0 || blocked || rq < 0) continue;
      if (rq == LFA_VARIANT_BLOCKED) {
        // an explicit request always takes the route; the autotuner cache's choice (timed on a
        // layer with many symbols) only when this layer has enough symbols to fill the GPU
        if (!p->plain && bj_supported(La.M, La.N) && (q == 0 || La.F_h >= bj_min_symbols(La.N))) blocked = true;
      } else if (rq & LFA_VARIANT_LOGGED) {
        const int id = rq & (LFA_VARIANT_LOGGED - 1);
        if (can_log && id < kNumVariants && logged_ok(id, La.M, La.N)) { v = id; logged = true; }
      } else if (variant_fits(rq, La.M, La.N, p->vec)) {
        v = rq;
      }
    }
    // built-in choice: the blocked tensor-core route for tall or square symbols of more than 128
    // columns, in layers with enough symbols to fill the GPU (bj_min_symbols); measured faster than
    // the element-wise kernels there, with and without vectors (at 192 columns, 514 symbols: 46 ms
    // against 167 ms with vectors). 128 columns: the autotuner cache decides
    if (v < 0 && !blocked && !p->plain && !La.wide && La.N > 128 && bj_supported(La.M, La.N) &&
        La.F_h >= bj_min_symbols(La.N))
      blocked = true;
    if (blocked) {
      int ctas = 0;
      cudaError_t be = bj_max_ctas(p->vec, prop.multiProcessorCount, &ctas);
      if (be != cudaSuccess || ctas < 1) { free_plan(p); return be != cudaSuccess ? from_cuda(be) : LFA_ERR_UNSUPPORTED; }
      p->blocked.push_back({l, ctas, 0});   // the CTA count is the launch's, set per group below
      p->variant[l] = -1;
    }
    if (!blocked && v < 0) v = choose_variant(La.M, La.N, p->vec);
    if (!blocked && v < 0 && can_log) {
      // W does not fit registers next to X: values-mode variant + rotation log + replay
      v = choose_variant(La.M, La.N, false);
      if (v >= 0 && logged_ok(v, La.M, La.N)) logged = true;
      else v = -1;
    }
    if (!blocked && v < 0) { free_plan(p); return LFA_ERR_UNSUPPORTED; }
    if (!blocked) p->variant[l] = v;
    if (logged) {
      lfa_plan_s::Logged lg;
      lg.layer = l;
      lg.variant = v;
      lg.grid = 0;
      lg.sweeps_cap = std::min(p->max_sweeps, 24);
      lg.log_cap = lg.sweeps_cap * (2 * kVariants[v].NP - 1);
      const size_t per_symbol = (size_t)lg.log_cap * kVariants[v].NP * sizeof(float4) +
                                (size_t)(La.M + La.N) * La.N * sizeof(float2);
      const size_t budget = (size_t)2 << 30;
      lg.batch = (int)std::max<size_t>(1, std::min<size_t>(budget / per_symbol, (size_t)La.F_h));
      log_bytes = std::max(log_bytes, (size_t)lg.batch * lg.log_cap * kVariants[v].NP * sizeof(float4));
      ranks_bytes = std::max(ranks_bytes, (size_t)lg.batch * La.M * La.N * sizeof(float2));    // raw X
      wraw_bytes = std::max(wraw_bytes, (size_t)lg.batch * La.N * La.N * sizeof(float2));
      rounds_bytes = std::max(rounds_bytes, (size_t)lg.batch * sizeof(int32_t));
      p->logged.push_back(lg);
    }
    off_half[l] = bytes; bytes += align256((size_t)La.F_h * 4);
    off_twn[l] = bytes; bytes += align256((size_t)d.n * 8);
    off_twm[l] = bytes; bytes += align256((size_t)d.m * 8);
    const size_t CC = (size_t)La.c_out * La.c_in;   // symbol entries
    if (p->plain) sym_bytes = std::max(sym_bytes, (size_t)La.F_h * CC * 8);
    if (p->vec) g_need = std::max(g_need, (size_t)La.F_h * CC * 8);
  }
  // backward workspace: G for at most 256 MB worth of symbols (at least one chunk)
  const size_t g_budget = (size_t)256 << 20;
  size_t g_bytes = 0;
  if (p->vec) {
    g_bytes = std::min(g_need, g_budget);
    for (int l = 0; l < nlayers; ++l) {
      const LayerArgs& La = p->args[l];
      const int64_t CC = (int64_t)La.c_out * La.c_in;
      if (La.F_h <= 0) { p->bw_chunks[l] = 1; continue; }   // an empty shard
      const int64_t cap = std::max<int64_t>(1, (int64_t)(g_bytes / (CC * 8)));
      int64_t chunks = std::max<int64_t>((155648 + CC - 1) / CC, (La.F_h + cap - 1) / cap);
      chunks = std::min<int64_t>(std::min<int64_t>(chunks, La.F_h), 4096);
      int64_t chunk = std::min<int64_t>((La.F_h + chunks - 1) / chunks, 65535);
      chunks = (La.F_h + chunk - 1) / chunk;
      g_bytes = std::max(g_bytes, (size_t)(chunk * CC * 8));
      const int fused = fused_backward_chunks(La);   // the fused backward picks its own chunking
      if (fused > 0) chunks = fused;
      const int tc_parts = tc_backward_parts(La);     // the tensor-core backward: its partial slabs
      if (tc_parts > 0) chunks = tc_parts;
      p->bw_chunks[l] = (int)chunks;
      part_bytes = std::max(part_bytes, (size_t)(chunks * CC * La.kh * La.kw * 4));
    }
  }
  // blocked launches: layers whose symbols pad to the same Mp x Np share one persistent launch
  for (int b = 0; b < (int)p->blocked.size(); ++b) {
    const LayerArgs& La = p->args[p->blocked[b].layer];
    int Mp = 0, Np = 0;
    bj_dims(La.M, La.N, &Mp, &Np);
    auto it = std::find_if(p->bj_groups.begin(), p->bj_groups.end(),
                           [&](const lfa_plan_s::BlockedGroup& g) { return g.Mp == Mp && g.Np == Np; });
    if (it == p->bj_groups.end()) {
      p->bj_groups.push_back({{b}, 0, Mp, Np, 0});
      it = p->bj_groups.end() - 1;
    } else {
      it->members.push_back(b);
    }
  }
  for (auto& g : p->bj_groups) {
    int items = 0;
    for (int b : g.members) items += p->args[p->blocked[b].layer].F_h;
    g.ctas = std::min(p->blocked[g.members[0]].ctas, std::max(1, items));
    if (g_bj_max_ctas > 0) g.ctas = std::min(g.ctas, g_bj_max_ctas);
    // warm starts (vectors): two runs of neighbouring symbols per CTA, so that the CTA taking a
    // run's next symbol finds the previous one done (about two symbol times apart in the queue)
    // (none with LFA_REPRODUCIBLE: whether a predecessor is done depends on timing)
    g.runs = (!p->vec || p->reproducible || g_bj_runs < 0) ? 0 : g_bj_runs > 0 ? g_bj_runs : 2 * g.ctas;
    for (int b : g.members) {
      p->blocked[b].ctas = g.ctas;
      p->blocked[b].sym_begin = p->bj_symbols;
      p->bj_symbols += p->args[p->blocked[b].layer].F_h;
    }
    bj_bytes = std::max(bj_bytes, (size_t)g.ctas * bj_slot_floats(g.Mp, g.Np, p->vec) * sizeof(float));
  }
  const size_t off_sym = bytes; bytes += align256(sym_bytes);
  const size_t off_g = bytes; bytes += align256(g_bytes);
  const size_t off_part = bytes; bytes += align256(part_bytes);
  size_t edit_bytes = 0;
  if (p->vec)
    for (int l = 0; l < nlayers; ++l)
      edit_bytes = std::max(edit_bytes, (size_t)(p->half_output ? p->args[l].F_h : p->args[l].n * p->args[l].m) *
                                            p->args[l].r * sizeof(float));
  const size_t off_edit = bytes; bytes += align256(edit_bytes);
  const size_t off_reg = bytes; bytes += align256(kRegScratchBytes);
  const size_t off_log = bytes; bytes += align256(log_bytes);
  const size_t off_ranks = bytes; bytes += align256(ranks_bytes);
  const size_t off_rounds = bytes; bytes += align256(rounds_bytes);
  const size_t off_wraw = bytes; bytes += align256(wraw_bytes);
  const size_t off_bj = bytes; bytes += align256(bj_bytes);
  const size_t off_done = bytes; bytes += align256((size_t)p->bj_symbols * sizeof(int32_t));
  // FFT route: transform batches of channel pairs within 512 MB of real grids and spectra
  size_t fft_bytes = 0;
  if (p->fft) {
    p->fft_pairs.assign(nlayers, 0);
    p->fft_plans.assign(nlayers, nullptr);
    for (int l = 0; l < nlayers; ++l) {
      const LayerArgs& La = p->args[l];
      const int pairs = std::max(1, fft_chunk_pairs(La, (size_t)512 << 20));
      p->fft_pairs[l] = pairs;
      fft_bytes = std::max(fft_bytes, (size_t)pairs * ((size_t)La.n * La.m * 4 + (size_t)La.n * (La.m / 2 + 1) * 8));
    }
  }
  const size_t off_fft = bytes; bytes += align256(fft_bytes);

  cudaError_t e = cudaMalloc(&p->dmem, bytes);
  if (e != cudaSuccess) { free_plan(p); return from_cuda(e); }
  p->dbytes = bytes;
  char* base = static_cast<char*>(p->dmem);
  p->counters = reinterpret_cast<Counters*>(base);
  p->sym_ws = sym_bytes ? reinterpret_cast<float2*>(base + off_sym) : nullptr;
  p->g_ws = g_bytes ? reinterpret_cast<float2*>(base + off_g) : nullptr;
  p->g_cap_bytes = (int64_t)g_bytes;
  p->partial_ws = part_bytes ? reinterpret_cast<float*>(base + off_part) : nullptr;
  p->edit_ws = edit_bytes ? reinterpret_cast<float*>(base + off_edit) : nullptr;
  p->reg_ws = reinterpret_cast<float*>(base + off_reg);
  p->log_ws = log_bytes ? reinterpret_cast<float4*>(base + off_log) : nullptr;
  p->xraw_ws = ranks_bytes ? reinterpret_cast<float2*>(base + off_ranks) : nullptr;
  p->rounds_ws = rounds_bytes ? reinterpret_cast<int32_t*>(base + off_rounds) : nullptr;
  p->wraw_ws = wraw_bytes ? reinterpret_cast<float2*>(base + off_wraw) : nullptr;
  p->bj_ws = bj_bytes ? reinterpret_cast<float*>(base + off_bj) : nullptr;
  p->bj_done = p->bj_symbols ? reinterpret_cast<int32_t*>(base + off_done) : nullptr;
  p->fft_ws = fft_bytes ? static_cast<void*>(base + off_fft) : nullptr;
  for (int l = 0; l < nlayers && p->fft && e == cudaSuccess; ++l)
    e = fft_make_plan(p->args[l], p->fft_pairs[l], &p->fft_plans[l]);

  // ---- upload tables (synchronous, plan time only)
  std::vector<float2> tw;
  auto twiddles = [&](int n) {
    tw.resize(n);
    for (int t = 0; t < n; ++t) {
      // exp(2 pi i t / n) in fp64 with exact integer reduction, rounded to fp32 once
      const double ang = 6.283185307179586476925286766559 * (double)t / (double)n;
      tw[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  };
  for (int l = 0; l < nlayers && e == cudaSuccess; ++l) {
    LayerArgs& La = p->args[l];
    La.half = reinterpret_cast<const int32_t*>(base + off_half[l]);
    La.tw_n = reinterpret_cast<const float2*>(base + off_twn[l]);
    La.tw_m = reinterpret_cast<const float2*>(base + off_twm[l]);
    La.dbg = &p->counters->debug_error;
    e = cudaMemcpy(base + off_half[l], p->half_host[l].data(), (size_t)La.F_h * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
    twiddles(La.n);
    e = cudaMemcpy(base + off_twn[l], tw.data(), (size_t)La.n * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
    twiddles(La.m);
    e = cudaMemcpy(base + off_twm[l], tw.data(), (size_t)La.m * 8, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(p->counters, 0, sizeof(Counters));
  // ---- variant groups (one persistent launch per variant) and kernel attributes
  for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v) {
    lfa_plan_s::Group g;
    g.variant = v;
    g.items = 0;
    for (int l = 0; l < nlayers; ++l)
      if (p->variant[l] == v && std::none_of(p->blocked.begin(), p->blocked.end(),
                                              [l](const lfa_plan_s::Blocked& q) { return q.layer == l; }) &&
          std::none_of(p->logged.begin(), p->logged.end(),
                                              [l](const lfa_plan_s::Logged& q) { return q.layer == l; })) {
        g.layers.push_back(l);
        g.items += (p->args[l].F_h + variant_spu(v) - 1) / variant_spu(v);
      }
    if (g.layers.empty()) continue;
    const bool fused = !p->plain;
    e = vprepare(v, p->vec, fused);
    if (e != cudaSuccess) break;
    int full = 0;
    e = vgrid(v, p->vec, fused, p->sms, &full);
    if (e != cudaSuccess) break;
    if (full < 1) { e = cudaErrorInvalidConfiguration; break; }
    // a persistent grid: no more CTAs than can be co-resident, none without an item
    const int cs = variant_cs(v);
    g.grid = std::max(cs, std::min(g.items * cs, full) / cs * cs);
    p->groups.push_back(g);
    if (p->plain)
      for (int l : g.layers) {
        const int items = (p->args[l].F_h + variant_spu(v) - 1) / variant_spu(v);
        p->plain_grid[l] = std::max(cs, std::min(items * cs, full) / cs * cs);
      }
  }
  for (auto& lg : p->logged) {
    if (e != cudaSuccess) break;
    e = jacobi_val_log_prepare(lg.variant);
    if (e == cudaSuccess) e = prepare_replay(kVariants[lg.variant].NP);
    if (e == cudaSuccess) e = jacobi_val_log_grid(lg.variant, p->sms, &lg.grid);
    if (e == cudaSuccess && lg.grid < 1) e = cudaErrorInvalidConfiguration;
  }
  if (e == cudaSuccess && p->groups.size() > 14) e = cudaErrorInvalidValue;   // 14: blocked, 15: logged layers
  if (e == cudaSuccess && p->use_graph) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  // streams and events of the forward's parallel parts
  const size_t nparts = p->groups.size() + (p->bj_groups.empty() ? 0 : 1) + (p->logged.empty() ? 0 : 1);
  if (e == cudaSuccess && !p->plain && nparts > 1) {
    e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    for (size_t k = 0; k < nparts && e == cudaSuccess; ++k) {
      cudaStream_t b = nullptr;
      cudaEvent_t j = nullptr;
      e = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking);
      if (e == cudaSuccess) p->branch.push_back(b);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
      if (e == cudaSuccess) p->join.push_back(j);
    }
  }
  if (e != cudaSuccess) { free_plan(p); return from_cuda(e); }
  *plan = p;
  return LFA_OK;
}

lfa_status_t lfa_svd(lfa_plan_t p, const float* const* w, float* const* sigma, float* const* U,
                     float* const* V, void* stream) {
  NvtxRange nvtx_range("lfa_svd");
  if (p == nullptr || w == nullptr || sigma == nullptr) return LFA_ERR_INVALID_ARG;
  if (p->vec && (U == nullptr || V == nullptr)) return LFA_ERR_INVALID_ARG;
  for (int l = 0; l < p->nlayers; ++l) {
    if (w[l] == nullptr || sigma[l] == nullptr) return LFA_ERR_INVALID_ARG;
    if (p->vec && (U[l] == nullptr || V[l] == nullptr)) return LFA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  p->last_stream = s;
  if (!p->use_graph) {
    lfa_status_t st = enqueue_forward(p, w, sigma, U, V, s);
    if (st == LFA_OK && !p->plain) g_launches += (int64_t)p->groups.size() + logged_launches(p);
    return st;
  }
  // graph path: capture once per distinct set of buffers, then replay
  std::vector<const void*> key;
  key.reserve(4 * p->nlayers);
  for (int l = 0; l < p->nlayers; ++l) {
    key.push_back(w[l]);
    key.push_back(sigma[l]);
    key.push_back(p->vec ? U[l] : nullptr);
    key.push_back(p->vec ? V[l] : nullptr);
  }
  if (p->exec == nullptr || key != p->graph_key) {
    if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
    if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    LFA_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    lfa_status_t st = enqueue_forward(p, w, sigma, U, V, p->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    if (st != LFA_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return from_cuda(e);
    p->graph = g;
    e = cudaGraphInstantiate(&p->exec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); p->graph = nullptr; p->exec = nullptr; return from_cuda(e); }
    p->graph_key = key;
  }
  lfa_status_t st = from_cuda(cudaGraphLaunch(p->exec, s));
  if (st == LFA_OK) g_launches += (int64_t)p->groups.size() + logged_launches(p);
  return st;
}

lfa_status_t lfa_symbols(lfa_plan_t p, int32_t layer, const float* w, float* out, void* stream) {
  if (p == nullptr || w == nullptr || out == nullptr || layer < 0 || layer >= p->nlayers)
    return LFA_ERR_INVALID_ARG;
  LayerArgs La = p->args[layer];
  La.w = w;
  g_launches += 1;
  return from_cuda(launch_symbols(La, reinterpret_cast<float2*>(out), static_cast<cudaStream_t>(stream)));
}

lfa_status_t lfa_fft_symbols(lfa_plan_t p, int32_t layer, const float* w, float* out, void* stream) {
  if (p == nullptr || !p->fft || w == nullptr || out == nullptr || layer < 0 || layer >= p->nlayers)
    return LFA_ERR_INVALID_ARG;
  LayerArgs La = p->args[layer];
  La.w = w;
  int nk = 0;
  const lfa_status_t st = from_cuda(launch_fft_symbols(La, p->fft_plans[layer], p->fft_pairs[layer], p->fft_ws,
                                                        reinterpret_cast<float2*>(out), static_cast<cudaStream_t>(stream),
                                                        &nk));
  g_launches += nk;
  return st;
}

lfa_status_t lfa_expand(lfa_plan_t p, int32_t layer, const float* U, const float* V, int64_t first,
                        int64_t count, float* u_hat, float* v_hat, void* stream) {
  NvtxRange nvtx_range("lfa_expand");
  if (p == nullptr || layer < 0 || layer >= p->nlayers || !p->vec) return LFA_ERR_INVALID_ARG;
  if (p->shard_count > 1) return LFA_ERR_UNSUPPORTED;
  const LayerArgs& La = p->args[layer];
  const int64_t total = (int64_t)La.n * La.m * La.r;
  if (first < 0 || count < 0 || first + count > total) return LFA_ERR_INVALID_ARG;
  if ((u_hat && !U) || (v_hat && !V)) return LFA_ERR_INVALID_ARG;
  // launch_expand splits a range into launches of at most 65535 groups of 32 vectors
  if (count > 0) g_launches += (count + 65535LL * 32 - 1) / (65535LL * 32);
  return from_cuda(launch_expand(La, reinterpret_cast<const float2*>(U), reinterpret_cast<const float2*>(V),
                                 first, count, reinterpret_cast<float2*>(u_hat),
                                 reinterpret_cast<float2*>(v_hat), static_cast<cudaStream_t>(stream)));
}

lfa_status_t lfa_svd_backward(lfa_plan_t p, const float* const* dsigma, const float* const* U,
                              const float* const* V, float* const* dw, void* stream) {
  NvtxRange nvtx_range("lfa_svd_backward");
  if (p == nullptr || !p->vec || dsigma == nullptr || U == nullptr || V == nullptr || dw == nullptr)
    return LFA_ERR_INVALID_ARG;
  for (int l = 0; l < p->nlayers; ++l)
    if (!dsigma[l] || !U[l] || !V[l] || !dw[l]) return LFA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every layer's backward in turn (they share the G and partial-sum workspaces)
  auto enqueue = [&](cudaStream_t st, int64_t* kernels) -> lfa_status_t {
    for (int l = 0; l < p->nlayers; ++l) {
      const LayerArgs& La = p->args[l];
      const int64_t CC = (int64_t)La.c_out * La.c_in;
      const int64_t g_cap = p->g_cap_bytes / (CC * 8);
      int nk = 0;
      LFA_CUDA_TRY(launch_backward(La, dsigma[l], p->half_output, reinterpret_cast<const float2*>(U[l]),
                                   reinterpret_cast<const float2*>(V[l]), p->g_ws, g_cap, p->partial_ws,
                                   p->bw_chunks[l], dw[l], st, &nk, p->counters->bw_queue, p->counters, p->sms));
      *kernels += nk;
    }
    return LFA_OK;
  };
  if (!p->use_graph) {
    int64_t nk = 0;
    const lfa_status_t st = enqueue(s, &nk);
    g_launches += nk;
    return st;
  }
  // graph path: capture once per distinct set of buffers, then replay
  std::vector<const void*> key;
  key.reserve(4 * p->nlayers);
  for (int l = 0; l < p->nlayers; ++l) {
    key.push_back(dsigma[l]);
    key.push_back(U[l]);
    key.push_back(V[l]);
    key.push_back(dw[l]);
  }
  if (p->bw_exec == nullptr || key != p->bw_key) {
    if (p->bw_exec) { cudaGraphExecDestroy(p->bw_exec); p->bw_exec = nullptr; }
    if (p->bw_graph) { cudaGraphDestroy(p->bw_graph); p->bw_graph = nullptr; }
    LFA_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    int64_t nk = 0;
    const lfa_status_t st = enqueue(p->cap_stream, &nk);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    if (st != LFA_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return from_cuda(e);
    p->bw_graph = g;
    e = cudaGraphInstantiate(&p->bw_exec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); p->bw_graph = nullptr; p->bw_exec = nullptr; return from_cuda(e); }
    p->bw_key = key;
    p->bw_kernels = nk;
  }
  const lfa_status_t st = from_cuda(cudaGraphLaunch(p->bw_exec, s));
  if (st == LFA_OK) g_launches += p->bw_kernels;
  return st;
}

lfa_status_t lfa_spectral_edit(lfa_plan_t p, const float* const* sigma, const float* const* U,
                               const float* const* V, int32_t mode, float a, float b, float* const* w_out,
                               void* stream) {
  if (p == nullptr || !p->vec || sigma == nullptr || U == nullptr || V == nullptr || w_out == nullptr)
    return LFA_ERR_INVALID_ARG;
  if (mode < LFA_EDIT_CLIP || mode > LFA_EDIT_PINV || !std::isfinite(a) || !std::isfinite(b)) return LFA_ERR_INVALID_ARG;
  for (int l = 0; l < p->nlayers; ++l) {
    if (!sigma[l] || !U[l] || !V[l] || !w_out[l]) return LFA_ERR_INVALID_ARG;
    if (mode == LFA_EDIT_PINV && (p->args[l].sh != 1 || p->args[l].sw != 1)) return LFA_ERR_UNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int l = 0; l < p->nlayers; ++l) {
    LayerArgs La = p->args[l];
    const float2* Ul = reinterpret_cast<const float2*>(U[l]);
    const float2* Vl = reinterpret_cast<const float2*>(V[l]);
    LFA_CUDA_TRY(launch_edit_values(La, p->half_output, sigma[l], mode, a, b, p->edit_ws, s));
    if (mode == LFA_EDIT_PINV) {
      // A^+ has the symbols V S^+ U^*: the backward of the transposed layer, U and V exchanged
      std::swap(La.c_out, La.c_in);
      La.c_w = La.c_in;
      La.wide = La.c_in > La.c_out ? 1 : 0;
      std::swap(Ul, Vl);
    }
    const int64_t CC = (int64_t)La.c_out * La.c_in;
    const int64_t g_cap = p->g_cap_bytes / (CC * 8);
    int nk = 0;
    LFA_CUDA_TRY(launch_backward(La, p->edit_ws, p->half_output, Ul, Vl, p->g_ws, g_cap, p->partial_ws,
                                 p->bw_chunks[l], w_out[l], s, &nk, p->counters->bw_queue, p->counters, p->sms));
    g_launches += 1 + nk;
  }
  return LFA_OK;
}

lfa_status_t lfa_regulariser_grad(lfa_plan_t p, const float* const* sigma, float lam,
                                  float* const* dsigma, float* const* loss, void* stream) {
  if (p == nullptr || sigma == nullptr || dsigma == nullptr || !std::isfinite(lam)) return LFA_ERR_INVALID_ARG;
  if (p->shard_count > 1) return LFA_ERR_UNSUPPORTED;
  for (int l = 0; l < p->nlayers; ++l)
    if (!sigma[l] || !dsigma[l]) return LFA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int l = 0; l < p->nlayers; ++l) {
    LFA_CUDA_TRY(launch_regulariser(p->args[l], p->half_output, sigma[l], lam, dsigma[l],
                                    loss ? loss[l] : nullptr, p->reg_ws, s));
    g_launches += 2;
  }
  return LFA_OK;
}

lfa_status_t lfa_destroy(lfa_plan_t p) {
  if (p == nullptr) return LFA_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_plan(p);
  return from_cuda(e);
}

lfa_status_t lfa_get_info(lfa_plan_t p, lfa_info_t* info) {
  if (p == nullptr || info == nullptr) return LFA_ERR_INVALID_ARG;
  LFA_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
  Counters c;
  LFA_CUDA_TRY(cudaMemcpy(&c, p->counters, sizeof c, cudaMemcpyDeviceToHost));
  std::memset(info, 0, sizeof *info);
  for (int l = 0; l < p->nlayers; ++l) {
    info->symbols += p->args[l].F_h;
    info->singular_values += p->shard_count > 1 ? 0 : (int64_t)p->args[l].n * p->args[l].m * p->args[l].r;
    if (p->shard_count > 1) {
      // the shard's frequencies: a half-grid frequency stands for itself and its conjugate
      for (int32_t f : p->half_host[l]) {
        const int j = f / p->args[l].m, ll = f - j * p->args[l].m;
        const int fc = ((p->args[l].n - j) % p->args[l].n) * p->args[l].m + (p->args[l].m - ll) % p->args[l].m;
        info->singular_values += (int64_t)(fc == f ? 1 : 2) * p->args[l].r;
      }
    }
  }
  info->unconverged = (int64_t)c.unconverged;
  info->nonfinite = (int64_t)c.nonfinite;
  info->sweeps = (int64_t)c.sweeps;
  info->rotations = (int64_t)c.rotations;
  info->plan_device_bytes = (int64_t)p->dbytes;
  info->nlayers = p->nlayers;
  info->max_sweeps = p->max_sweeps;
  info->tol = p->tol_opt > 0.f ? p->tol_opt : default_tol(p->args[0].M, p->args[0].wide != 0);
  info->tc_grams = (int64_t)c.tc_grams;
  info->tc_updates = (int64_t)c.tc_updates;
  info->debug_error = (int32_t)c.debug_error;
  if (c.debug_error) return LFA_ERR_CUDA;   // debug build: a kernel index left its range
  if (c.timeouts) return LFA_ERR_TIMEOUT;
  if (c.nonfinite) return LFA_ERR_NONFINITE;
  if (c.unconverged) return LFA_ERR_NOT_CONVERGED;
  return LFA_OK;
}

lfa_status_t lfa_layer_query(lfa_plan_t p, int32_t layer, int64_t* F_h, int32_t* r, int32_t* variant,
                             int32_t* half_grid) {
  if (p == nullptr || layer < 0 || layer >= p->nlayers) return LFA_ERR_INVALID_ARG;
  if (F_h) *F_h = p->args[layer].F_h;
  if (r) *r = p->args[layer].r;
  if (variant) {
    const bool logged = std::any_of(p->logged.begin(), p->logged.end(),
                                    [layer](const lfa_plan_s::Logged& q) { return q.layer == layer; });
    const bool blocked = std::any_of(p->blocked.begin(), p->blocked.end(),
                                     [layer](const lfa_plan_s::Blocked& q) { return q.layer == layer; });
    *variant = blocked ? LFA_VARIANT_BLOCKED : (p->variant[layer] | (logged ? LFA_VARIANT_LOGGED : 0));
  }
  if (half_grid) std::memcpy(half_grid, p->half_host[layer].data(), p->half_host[layer].size() * 4);
  return LFA_OK;
}

const char* lfa_status_string(lfa_status_t s) {
  switch (s) {
    case LFA_OK: return "ok";
    case LFA_ERR_INVALID_ARG: return "invalid argument";
    case LFA_ERR_UNSUPPORTED: return "unsupported";
    case LFA_ERR_OOM: return "out of memory";
    case LFA_ERR_CUDA: return "CUDA error";
    case LFA_ERR_NOT_CONVERGED: return "a symbol did not converge";
    case LFA_ERR_NONFINITE: return "non-finite input or result";
    case LFA_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

const char* lfa_variant_name(int32_t v) {
  if (v == LFA_VARIANT_BLOCKED) return "blocked_tc_b32";
  static const std::vector<std::string> logged_names = [] {
    std::vector<std::string> out;
    for (int i = 0; i < kNumVariants; ++i) out.push_back(std::string(kVariantNames[i]) + "_log");
    return out;
  }();
  if (v >= 0 && (v & LFA_VARIANT_LOGGED)) {
    const int id = v & (LFA_VARIANT_LOGGED - 1);
    return id < kNumVariants ? logged_names[id].c_str() : "none";
  }
  if (v < 0 || v >= kNumVariants) return "none";
  return kVariantNames[v];
}

int32_t lfa_last_cuda_error(void) { return g_last_cuda_error; }
int64_t lfa_kernel_launches(void) { return g_launches.load(); }
int32_t lfa_version(void) { return 100; }

// ----------------------------------------------------------------------------- host-logic hooks
int32_t lfa_debug_schedule(int32_t ncols, uint16_t* out, int64_t cap) {
  if (ncols < 2 || (ncols & 1) || ncols > 1024) return -1;
  std::vector<ushort2> s;
  if (!build_schedule(ncols, s)) return -2;
  if (out) {
    if ((int64_t)s.size() * 2 > cap) return -3;
    for (size_t i = 0; i < s.size(); ++i) { out[2 * i] = s[i].x; out[2 * i + 1] = s[i].y; }
  }
  return ncols - 1;
}

int64_t lfa_debug_half_grid(int32_t n, int32_t m, int32_t* out, int64_t cap) {
  if (n < 1 || m < 1 || (int64_t)n * m > 0x7fffffffLL) return -1;
  std::vector<int32_t> h;
  build_half_grid(n, m, h);
  if (out) {
    if ((int64_t)h.size() > cap) return -3;
    std::memcpy(out, h.data(), h.size() * 4);
  }
  return (int64_t)h.size();
}

int32_t lfa_debug_choose_variant(int32_t M, int32_t N, int32_t vectors) {
  return choose_variant(M, N, vectors != 0);
}

int32_t lfa_debug_variant_count(void) { return kNumVariants; }

int32_t lfa_debug_tuned_variant(const char* path, int32_t M, int32_t N, int32_t vectors) {
  return tuned_variant(path, M, N, vectors != 0);
}

int64_t lfa_debug_half_position(int32_t n, int32_t m, int32_t f) {
  if (n < 1 || m < 1 || (int64_t)n * m > 0x7fffffffLL || f < 0 || (int64_t)f >= (int64_t)n * m) return -1;
  return half_position(n, m, f);
}

int32_t lfa_debug_variant_fits(int32_t v, int32_t M, int32_t N, int32_t vectors) {
  return variant_fits(v, M, N, vectors != 0) ? 1 : 0;
}

int64_t lfa_debug_shard_range(int32_t n, int32_t m, int32_t rank, int32_t count_shards, int64_t* first,
                              int64_t* count) {
  if (n < 1 || m < 1 || (int64_t)n * m > 0x7fffffffLL || count_shards < 1 || count_shards > 65536 || rank < 0 ||
      rank >= count_shards || first == nullptr || count == nullptr)
    return -1;
  const int64_t s = (1 + (n % 2 == 0)) * (1 + (m % 2 == 0));
  const int64_t F_h = ((int64_t)n * m + s) / 2;
  shard_range(F_h, rank, count_shards, first, count);
  return F_h;
}

int32_t lfa_debug_backward_route(int32_t c_out, int32_t c_in, int32_t kh, int32_t kw, int32_t stride_h,
                                 int32_t stride_w) {
  LayerArgs La;
  std::memset(&La, 0, sizeof La);
  if (!set_geometry(La, c_out, c_in, kh, kw, 8, 8, -1, -1, stride_h, stride_w)) return -1;
  La.F_h = 1;
  if (tc_backward_parts(La) > 0) return 2;
  return fused_backward_chunks(La) > 0 ? 1 : 0;
}

int32_t lfa_debug_bj_profile(void* plan, uint64_t* out, int32_t* ctas) {
  lfa_plan_s* p = static_cast<lfa_plan_s*>(plan);
  if (p == nullptr || out == nullptr || ctas == nullptr) return LFA_ERR_INVALID_ARG;
  LFA_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
  Counters c;
  LFA_CUDA_TRY(cudaMemcpy(&c, p->counters, sizeof c, cudaMemcpyDeviceToHost));
  for (int k = 0; k < 6; ++k) out[k] = (uint64_t)c.bj_cycles[k];
  out[6] = (uint64_t)c.warm_starts;
  *ctas = p->blocked.empty() ? 0 : p->blocked[0].ctas;
  return LFA_OK;
}

void lfa_debug_set_bj_ctas_per_sm(int32_t n) { g_bj_ctas_per_sm = n < 0 ? 0 : n; }

void lfa_debug_set_bj_grid(int32_t max_ctas, int32_t runs) {
  g_bj_max_ctas = max_ctas < 0 ? 0 : max_ctas;
  g_bj_runs = runs;
}

int32_t lfa_debug_bj_occupancy(int32_t vectors, int32_t* out) {
  if (out == nullptr) return LFA_ERR_INVALID_ARG;
  int b[2] = {0, 0}, r = 0, ss = 0, sd = 0;
  LFA_CUDA_TRY(bj_occupancy(vectors != 0, b, &r, &ss, &sd));
  out[0] = b[0];
  out[1] = r;
  out[2] = ss;
  out[3] = sd;
  out[4] = b[1];
  return LFA_OK;
}

int32_t lfa_debug_logged_ok(int32_t v, int32_t M, int32_t N) {
  return v >= 0 && v < kNumVariants && logged_ok(v, M, N) ? 1 : 0;
}

}  // extern "C"
