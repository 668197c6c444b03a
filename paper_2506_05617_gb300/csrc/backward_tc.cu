// The backward pass dL/dw of the LFA SVD on the tcgen05 tensor cores, for stride-1 layers of 128
// channels and more (arXiv 2506.05617, Sec. III: sigma_k are the singular values of the symbols
// A_k = sum_y M_y exp(2 pi i <k, y>); d sigma = Re(u^* dA v)). Two stages per block of half-grid
// frequencies:
//  1. G_h = U_h diag(g~_h) V_h^* (c_out x c_in complex) for every h of the block: a batched complex
//     GEMM, here as real products on the tensor cores with TF32 operands split in three (hi*hi +
//     hi*lo + lo*hi, FP32 accumulation in tensor memory), which keeps FP32 accuracy:
//       Re G = (g Ur) Vr^T + (g Ui) Vi^T,   Im G = (g Ui) Vr^T - (g Ur) Vi^T.
//     One CTA (256 threads, two per SM) takes output tiles of 128 x 128 (o, i) entries of one h at a
//     time from a persistent item list; the singular index s is the K dimension, staged 8 at a time
//     by the CTA's threads (rows scaled by g~, split into TF32 hi and lo) in K-major core matrices,
//     three chunk buffers deep; one thread issues the MMAs; the finished tile leaves tensor memory
//     through tcgen05.ld and is written to the G workspace.
//  2. partial[p][o][i][a][b] (+)= sum_h Re(G_h[o, i] exp(-2 pi i <k_h, y_ab>)) over part p of the
//     block: E entries per thread, the taps in registers, the phases of 32 frequencies at a time in
//     shared memory. Parts accumulate over the blocks in launch order, and a final kernel adds the
//     parts in order: deterministic.
#include "lfa_internal.cuh"
#include "tc_ptx.cuh"

namespace lfa {
namespace bwtc {

constexpr int THREADS = 256;
constexpr int TM = 128;                  // output rows (o) per tile: M of the MMA
constexpr int TN = 128;                  // output columns (i) per tile: N of the MMA
constexpr int KS = 8;                    // singular indices per chunk: K of one MMA
constexpr int NB = 3;                    // chunk buffers
constexpr int PD = 2;                    // chunks whose loads are in flight
constexpr uint32_t PART = TM * KS * 4;   // 4 KB: one operand part (hi or lo of one plane)
constexpr uint32_t BUF = 8 * PART;       // P hi | P lo | Qm hi | Qm lo | Vr hi | Vr lo | Vi hi | Vi lo
constexpr uint32_t TMEM_COLS = 256;      // Re G (128 columns) | Im G (128 columns)
constexpr uint32_t WAIT_LIMIT = 1u << 22;
constexpr int OFF_MISC = NB * BUF;
constexpr int SMEM = OFF_MISC + 128;
static_assert(TM == TN && THREADS == 2 * TM, "one staging thread per (row, half chunk) of both operands");

struct Misc {
  uint64_t mbar[NB + 1];   // [b]: the MMAs that read buffer b completed; [NB]: a tile's MMAs completed
  uint32_t tmem;
  int32_t failed;          // a bounded wait ran out: no further tensor work in this CTA
  int32_t item;
};
static_assert(sizeof(Misc) <= 128, "misc block");

__device__ __forceinline__ Misc* misc(unsigned char* sm) { return reinterpret_cast<Misc*>(sm + OFF_MISC); }

// Next phase of mbarrier b; bit b of ph is this thread's parity for it (every thread waits on every
// phase). A wait that runs out marks the CTA failed and counts a timeout; the CTA then issues no
// tensor work and skips later waits, but keeps its place in every barrier.
__device__ __forceinline__ void wait_bar(Misc* ms, Counters* ctr, int b, uint32_t& ph) {
  if (!*reinterpret_cast<volatile int32_t*>(&ms->failed)) {
    if (!tc::mbar_wait_bounded(&ms->mbar[b], (ph >> b) & 1u, WAIT_LIMIT))
      if (atomicExch(&ms->failed, 1) == 0 && ctr) atomicAdd(&ctr->timeouts, 1ull);
  }
  ph ^= 1u << b;
  tc::fence_after_sync();
}

}  // namespace bwtc

// Stage 1: G[h - h_begin][o][i] for h in [h_begin, h_end), every (o, i). Items are (h, o tile, i tile),
// h-major, pulled from counter `queue`.
__global__ void __launch_bounds__(bwtc::THREADS, 2)
bw_g_tc_kernel(LayerArgs La, const float* dsigma, int half_output, const float2* U, const float2* V, int h_begin,
               int h_end, float2* G, unsigned int* queue, Counters* ctr) {
  using namespace bwtc;
  extern __shared__ __align__(1024) unsigned char sm[];
  Misc* ms = misc(sm);
  const int co = La.c_out, ci = La.c_in, r = La.r;
  const int to = (co + TM - 1) / TM, ti = (ci + TN - 1) / TN;
  const int total = (h_end - h_begin) * to * ti;
  const int nch = (r + KS - 1) / KS;
  if (threadIdx.x == 0) {
    for (int k = 0; k <= NB; ++k) tc::mbar_init(&ms->mbar[k], 1);
    tc::fence_mbar_init();
    ms->failed = 0;
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(&ms->tmem, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  uint32_t ph = 0;
  const uint32_t s_base = tc::smem_u32(sm);
  const int row = threadIdx.x & (TM - 1);
  const int kc = threadIdx.x >> 7;          // this thread's quad of singular indices within a chunk
  const int soff = ((kc * 16 + (row >> 3)) * 8 + (row & 7)) * 4;
  constexpr uint32_t LBO = 2048, SBO = 128;
  constexpr uint32_t ID = tc::idesc_tf32(TM, TN);
  constexpr uint32_t ID_NEG = tc::idesc_tf32(TM, TN, false, true);

  for (;;) {
    if (threadIdx.x == 0) ms->item = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int it = ms->item;
    if (it >= total) break;
    const int h = h_begin + it / (to * ti);
    if (!LFA_DOK(La.dbg, h < h_end && h < La.F_h, 9)) {   // tensor-core G: item -> symbol
      __syncthreads();                                     // every thread has read ms->item
      continue;
    }
    const int tile = it % (to * ti);
    const int o0 = (tile / ti) * TM, i0 = (tile % ti) * TN;
    const int f = La.half[h];
    const int j = f / La.m, l = f - j * La.m;
    const int fc = ((La.n - j) % La.n) * La.m + (La.m - l) % La.m;
    const float* g_f = dsigma + (size_t)(half_output ? h : f) * r;
    const float* g_c = (!half_output && fc != f) ? dsigma + (size_t)fc * r : nullptr;
    const bool orow = o0 + row < co, irow = i0 + row < ci;
    const float2* Ur = U + ((size_t)h * co + (orow ? o0 + row : 0)) * r;
    const float2* Vr = V + ((size_t)h * ci + (irow ? i0 + row : 0)) * r;
    // a chunk's four singular indices of this thread: g~ U and V entries of its rows
    float2 pu[PD][4], pv[PD][4];
    // With r a multiple of 4 (and 16-byte aligned arrays), a thread's four singular indices are all in
    // range or all out, and its rows of U, V and dsigma start on 16-byte boundaries: 16-byte loads.
    const bool vec4 = (r & 3) == 0 && ((reinterpret_cast<uintptr_t>(dsigma) | reinterpret_cast<uintptr_t>(U) |
                                         reinterpret_cast<uintptr_t>(V)) & 15) == 0;
    auto prefetch = [&](int c, float2* u, float2* v) {
      const int s0 = c * KS + 4 * kc;
      if (vec4) {
        if (s0 < r) {
          float4 g4 = *reinterpret_cast<const float4*>(g_f + s0);
          if (g_c) {
            const float4 c4 = *reinterpret_cast<const float4*>(g_c + s0);
            g4 = make_float4(g4.x + c4.x, g4.y + c4.y, g4.z + c4.z, g4.w + c4.w);
          }
          const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 u01 = orow ? *reinterpret_cast<const float4*>(Ur + s0) : z;
          const float4 u23 = orow ? *reinterpret_cast<const float4*>(Ur + s0 + 2) : z;
          const float4 v01 = irow ? *reinterpret_cast<const float4*>(Vr + s0) : z;
          const float4 v23 = irow ? *reinterpret_cast<const float4*>(Vr + s0 + 2) : z;
          u[0] = make_float2(u01.x * g4.x, u01.y * g4.x);
          u[1] = make_float2(u01.z * g4.y, u01.w * g4.y);
          u[2] = make_float2(u23.x * g4.z, u23.y * g4.z);
          u[3] = make_float2(u23.z * g4.w, u23.w * g4.w);
          v[0] = make_float2(v01.x, v01.y);
          v[1] = make_float2(v01.z, v01.w);
          v[2] = make_float2(v23.x, v23.y);
          v[3] = make_float2(v23.z, v23.w);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) u[q] = v[q] = make_float2(0.f, 0.f);
        }
        return;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int s = s0 + q;
        const bool ok = s < r;
        const float g = ok ? g_f[s] + (g_c ? g_c[s] : 0.f) : 0.f;
        float2 x = (ok && orow) ? Ur[s] : make_float2(0.f, 0.f);
        u[q] = make_float2(x.x * g, x.y * g);
        v[q] = (ok && irow) ? Vr[s] : make_float2(0.f, 0.f);
      }
    };
    auto store_split = [&](float* st, float a, float b, float c, float d) {   // hi at st, lo one part on
      float4 hi, lo;
      tc::split_tf32(a, hi.x, lo.x);
      tc::split_tf32(b, hi.y, lo.y);
      tc::split_tf32(c, hi.z, lo.z);
      tc::split_tf32(d, hi.w, lo.w);
      *reinterpret_cast<float4*>(st + soff) = hi;
      *reinterpret_cast<float4*>(st + PART / 4 + soff) = lo;
    };
#pragma unroll
    for (int k = 0; k < PD; ++k)
      if (k < nch) prefetch(k, pu[k], pv[k]);
    for (int c0 = 0; c0 < nch; c0 += PD) {
#pragma unroll
      for (int k = 0; k < PD; ++k) {
        const int c = c0 + k;
        if (c >= nch) break;                              // uniform over the CTA
        const int b = c % NB;
        if (c >= NB) wait_bar(ms, ctr, b, ph);            // the MMAs of chunk c - NB released buffer b
        float* st = reinterpret_cast<float*>(sm + b * BUF);
        store_split(st, pu[k][0].x, pu[k][1].x, pu[k][2].x, pu[k][3].x);                 // P = g~ Re U
        store_split(st + 2 * PART / 4, pu[k][0].y, pu[k][1].y, pu[k][2].y, pu[k][3].y);  // Qm = g~ Im U
        store_split(st + 4 * PART / 4, pv[k][0].x, pv[k][1].x, pv[k][2].x, pv[k][3].x);  // Re V
        store_split(st + 6 * PART / 4, pv[k][0].y, pv[k][1].y, pv[k][2].y, pv[k][3].y);  // Im V
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (c + PD < nch) prefetch(c + PD, pu[k], pv[k]);
        if (threadIdx.x == 0 && !ms->failed) {
          tc::fence_after_sync();
          const uint32_t a0 = s_base + (uint32_t)b * BUF;
          const uint64_t ph_ = tc::smem_desc_kmajor(a0, LBO, SBO);
          const uint64_t pl_ = tc::smem_desc_kmajor(a0 + PART, LBO, SBO);
          const uint64_t qh_ = tc::smem_desc_kmajor(a0 + 2 * PART, LBO, SBO);
          const uint64_t ql_ = tc::smem_desc_kmajor(a0 + 3 * PART, LBO, SBO);
          const uint64_t rh_ = tc::smem_desc_kmajor(a0 + 4 * PART, LBO, SBO);
          const uint64_t rl_ = tc::smem_desc_kmajor(a0 + 5 * PART, LBO, SBO);
          const uint64_t ih_ = tc::smem_desc_kmajor(a0 + 6 * PART, LBO, SBO);
          const uint64_t il_ = tc::smem_desc_kmajor(a0 + 7 * PART, LBO, SBO);
          const uint32_t dre = ms->tmem, dim = ms->tmem + TN;
          const uint32_t acc0 = c > 0 ? 1u : 0u;
          // Re G += P Vr^T + Qm Vi^T
          tc::mma_tf32(dre, ph_, rh_, ID, acc0);
          tc::mma_tf32(dre, ph_, rl_, ID, 1u);
          tc::mma_tf32(dre, pl_, rh_, ID, 1u);
          tc::mma_tf32(dre, qh_, ih_, ID, 1u);
          tc::mma_tf32(dre, qh_, il_, ID, 1u);
          tc::mma_tf32(dre, ql_, ih_, ID, 1u);
          // Im G += Qm Vr^T - P Vi^T
          tc::mma_tf32(dim, qh_, rh_, ID, acc0);
          tc::mma_tf32(dim, qh_, rl_, ID, 1u);
          tc::mma_tf32(dim, ql_, rh_, ID, 1u);
          tc::mma_tf32(dim, ph_, ih_, ID_NEG, 1u);
          tc::mma_tf32(dim, ph_, il_, ID_NEG, 1u);
          tc::mma_tf32(dim, pl_, ih_, ID_NEG, 1u);
          tc::mma_commit(&ms->mbar[b]);
          if (c == nch - 1) tc::mma_commit(&ms->mbar[NB]);
        }
      }
    }
    wait_bar(ms, ctr, NB, ph);                            // every MMA of the tile completed
    // the buffers' last commits of this tile (already complete): one wait per commit keeps the parities
    for (int c = nch > NB ? nch - NB : 0; c < nch; ++c) wait_bar(ms, ctr, c % NB, ph);
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows o) and the columns [64 (w / 4), + 64) of
    // Re G and Im G
    {
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
      const int o = o0 + 32 * (w & 3) + lane;
      const int ib = i0 + 64 * (w >> 2);
      const uint32_t ta = ms->tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(64 * (w >> 2));
      float2* Go = G + ((size_t)(h - h_begin) * co + (o < co ? o : 0)) * ci;
#pragma unroll 1
      for (int g = 0; g < 4; ++g) {
        float re[16], im[16];
        tc::tmem_ld16(ta + 16 * g, re);
        tc::tmem_ld16(ta + TN + 16 * g, im);
        tc::tmem_ld_wait();
        if (o < co) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int i = ib + 16 * g + q;
            if (i < ci) Go[i] = make_float2(re[q], im[q]);
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();                                      // the accumulators are free for the next tile
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(ms->tmem, TMEM_COLS);
  }
}

// Stage 2 (stride 1): E consecutive (o, i) entries per thread; part p of [h_begin, h_end) (blockIdx.y)
// sums Re(G_h[o, i] conj(P_h[a, b])) over its frequencies in order and writes (accumulate = 0) or adds
// (accumulate = 1) partial[p][o][i][a][b].
template <int KK, int E>
__global__ void __launch_bounds__(256) bw_dw_tc_kernel(LayerArgs La, const float2* G, int h_begin, int h_end,
                                                      int nparts, int accumulate, float* partial) {
  constexpr int HB = 32;                  // frequencies whose phases are staged at once
  __shared__ float2 sph[HB][KK];
  const int CC = La.c_out * La.c_in;
  const int kk = La.kh * La.kw;
  const int e0 = (blockIdx.x * blockDim.x + threadIdx.x) * E;
  const int p = blockIdx.y;
  if (!LFA_DOK(La.dbg, p < nparts && h_end <= La.F_h, 10)) return;   // tap projection: part, range
  const int nh = h_end - h_begin;
  const int len = (nh + nparts - 1) / nparts;
  const int p0 = h_begin + p * len;
  const int p1 = min(h_end, p0 + len);
  float acc[E][KK];
#pragma unroll
  for (int q = 0; q < E; ++q)
#pragma unroll
    for (int t = 0; t < KK; ++t) acc[q][t] = 0.f;
  for (int hb = p0; hb < p1; hb += HB) {
    const int cnt = min(HB, p1 - hb);
    __syncthreads();
    for (int x = threadIdx.x; x < cnt * kk; x += blockDim.x) {
      const int hh = x / kk, t = x - hh * kk;
      const int f = La.half[hb + hh];
      const int j = f / La.m, l = f - j * La.m;
      sph[hh][t] = tap_phase(La, j, l, t / La.kw, t % La.kw);
    }
    __syncthreads();
    for (int hh = 0; hh < cnt; ++hh) {
      const float2* Gh = G + (size_t)(hb + hh - h_begin) * CC;
      float2 g[E];
#pragma unroll
      for (int q = 0; q < E; ++q) g[q] = e0 + q < CC ? Gh[e0 + q] : make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < KK; ++t) {
        if (t < kk) {
          const float2 ph = sph[hh][t];
#pragma unroll
          for (int q = 0; q < E; ++q) acc[q][t] = fmaf(g[q].x, ph.x, fmaf(g[q].y, ph.y, acc[q][t]));  // Re(g conj(ph))
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int e = e0 + q;
    if (e >= CC) continue;
    float* pp = partial + ((size_t)p * CC + e) * kk;
#pragma unroll
    for (int t = 0; t < KK; ++t)
      if (t < kk) pp[t] = accumulate ? pp[t] + acc[q][t] : acc[q][t];
  }
}

int tc_backward_parts(const LayerArgs& La) {
  if (La.sh != 1 || La.sw != 1 || La.c_out < 128 || La.c_in < 128 || La.kh * La.kw > 25 || La.F_h <= 0) return 0;
  return 4;
}

static cudaError_t bw_tc_prepare(int sms, int* ctas) {
  cudaError_t e = cudaFuncSetAttribute(bw_g_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bwtc::SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(bw_g_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  *ctas = 2 * sms;   // two CTAs of 256 threads per SM, each with half of the tensor memory
  return e;
}

cudaError_t launch_backward_tc(const LayerArgs& La, const float* dsigma, int half_output, const float2* U,
                               const float2* V, float2* G, int64_t g_cap, float* partial, int parts,
                               unsigned int* queue, Counters* ctr, float* dw, int sms, cudaStream_t s,
                               int* nkernels) {
  *nkernels = 0;
  const int kk = La.kh * La.kw;
  const int64_t CC = (int64_t)La.c_out * La.c_in;
  if (g_cap < 1 || parts < 1 || parts > 65535) return cudaErrorInvalidValue;
  int ctas = 0;
  cudaError_t e = bw_tc_prepare(sms, &ctas);
  if (e != cudaSuccess) return e;
  const int tiles = ((La.c_out + bwtc::TM - 1) / bwtc::TM) * ((La.c_in + bwtc::TN - 1) / bwtc::TN);
  const int per_block = (int)(g_cap < (int64_t)La.F_h ? g_cap : La.F_h);
  int slot = 0;
  for (int h0 = 0; h0 < La.F_h; h0 += per_block, ++slot) {
    const int h1 = h0 + per_block < La.F_h ? h0 + per_block : La.F_h;
    unsigned int* q = queue + (slot & 1);
    e = cudaMemsetAsync(q, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int items = (h1 - h0) * tiles;
    const int grid = items < ctas ? items : ctas;
    bw_g_tc_kernel<<<grid, bwtc::THREADS, bwtc::SMEM, s>>>(La, dsigma, half_output, U, V, h0, h1, G, q, ctr);
    ++*nkernels;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int acc = h0 > 0 ? 1 : 0;
    if (kk <= 1) {
      dim3 gd((unsigned)((CC + 256 * 4 - 1) / (256 * 4)), parts);
      bw_dw_tc_kernel<1, 4><<<gd, 256, 0, s>>>(La, G, h0, h1, parts, acc, partial);
    } else if (kk <= 9) {
      dim3 gd((unsigned)((CC + 256 * 4 - 1) / (256 * 4)), parts);
      bw_dw_tc_kernel<9, 4><<<gd, 256, 0, s>>>(La, G, h0, h1, parts, acc, partial);
    } else {
      dim3 gd((unsigned)((CC + 256 * 2 - 1) / (256 * 2)), parts);
      bw_dw_tc_kernel<25, 2><<<gd, 256, 0, s>>>(La, G, h0, h1, parts, acc, partial);
    }
    ++*nkernels;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t total = CC * kk;
  e = launch_backward_reduce(partial, parts, total, dw, s);
  ++*nkernels;
  return e;
}

}  // namespace lfa
