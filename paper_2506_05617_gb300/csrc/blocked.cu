// Blocked one-sided Jacobi SVD of large LFA symbols on the tcgen05 tensor cores (arXiv 2506.05617,
// Sec. III: the SVD A_k = U_k S_k V_k^* of each symbol, Algorithm 1 line 5), for symbols whose
// element-wise Jacobi is far from the FP32 roofline (c >= 128).
//
// Method (Hestenes' one-sided Jacobi, applied to blocks of columns): X = A_k (or A_k^* for wide
// symbols) has its N columns split into nb blocks of 32. A sweep visits every pair of blocks
// (I, J) once, in the circle-method order over blocks (nb / 2 disjoint pairs per round). For a
// pair, Y = [X_I, X_J] (M x 64) gives the Hermitian Gram matrix H = Y^* Y (64 x 64); one cyclic
// two-sided Jacobi sweep over H (63 rounds of 32 disjoint 2x2 rotations, each rotation chosen
// only when |h_pq| > tol sqrt(h_pp h_qq), the one-sided test) accumulates the unitary Q, and Y
// and the matching columns of W (the accumulated right factor, W = I initially) are replaced
// by Y Q and W Q. Because X = A W holds for any right factor, x_c = A w_c stays exact to
// rounding; sweeps repeat until no pair of a sweep rotates. Then sigma_c = |x_c| / |w_c|, the X
// columns normalised give U (V for wide symbols) and the W columns V (U).
//
// GB300 mapping:
//  * The two dense contractions of a block pair run on the tensor cores with TF32 operands
//    split 3 ways (hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor memory), which keeps
//    FP32 accuracy: the Gram in real form, Z^T Z with Z = [Re Y, Im Y] (M x 128, one
//    128 x 128 MMA tile, K = M), and the update Y Q in real form, [Re Y, Im Y] against Re Q
//    and Im Q (M = 128-row tiles, N = 64, K = 64, the negation of Im Q taken by the
//    instruction descriptor). Operands are staged by the CTA's threads (which split fp32 into
//    TF32 pairs) in K-major core-matrix layout; one thread issues the MMAs and an mbarrier
//    reports their completion.
//  * The inner 64 x 64 problem runs on the CUDA cores from shared memory.
//  * One thread-block cluster of nb / 2 CTAs works on one symbol: CTA i takes the block pair at
//    position i of each round, the cluster barrier separates rounds, and the symbol's X and W
//    (4 MB at 512 x 512) stay in L2 between rounds. Two CTAs per SM let one CTA's tensor work
//    overlap the other's inner problem. Clusters pull symbols from an atomic work queue.
#include <cooperative_groups.h>

#include <algorithm>

#include "jacobi.cuh"
#include "lfa_internal.cuh"
#include "tc_ptx.cuh"

namespace lfa {

namespace cg = cooperative_groups;

namespace bj {

constexpr int B = 32;            // columns per block
constexpr int P = 2 * B;         // columns of a block pair
constexpr int THREADS = 256;
constexpr int KC = 32;           // rows of X per Gram chunk (K of the Gram)
constexpr int RT = 128;          // rows of X (or W) per update tile (M of the update)
constexpr int KU = 16;           // columns of Y per update chunk (K of the update)
constexpr uint32_t TMEM_COLS = 128;
constexpr uint32_t WAIT_LIMIT = 1u << 22;

// shared memory (bytes)
constexpr int HS = P + 1;                            // row stride of H (float2): rows 520 B apart, so a
                                                     // column of H spreads over the shared-memory banks
constexpr int STAGE_BYTES = 33792;                   // Gram chunk hi|lo, update chunk, or H (64 x 65 float2)
constexpr int R1_BYTES = 65536;                      // Q (fp32) during the inner sweep, Q^T hi/lo after
constexpr int OFF_STAGE = 0;
constexpr int OFF_R1 = OFF_STAGE + STAGE_BYTES;
constexpr int OFF_PRM = OFF_R1 + R1_BYTES;           // float4 [32] rotation parameters
constexpr int OFF_TRI = OFF_PRM + 32 * 16;           // uint16 [528] block-pair (P, P') table
constexpr int OFF_PHS = OFF_TRI + 1056 + 32;          // float2 [256] phases of the symbol
constexpr int OFF_MISC = OFF_PHS + kMaxTaps * 8;     // mbarrier, tmem base, flags
constexpr int SMEM = OFF_MISC + 64;
static_assert(P * HS * 8 <= STAGE_BYTES, "H fits the staging area");
static_assert(OFF_R1 % 1024 == 0 && OFF_PRM % 16 == 0 && OFF_PHS % 16 == 0 && OFF_MISC % 16 == 0, "alignment");

struct Misc {
  uint64_t mbar;        // MMA completion
  uint32_t tmem;        // TMEM base column address
  uint32_t phase;       // parity of the next mbarrier phase
  int32_t rotated;      // the block pair rotated in its inner sweep
  int32_t failed;       // a bounded wait ran out: no further tensor work in this CTA
  int32_t item;         // work item (cluster rank 0)
  int32_t vote[2];      // sweep votes (cluster rank 0)
  int32_t pad[7];
};
static_assert(sizeof(Misc) <= 64, "misc block");

__device__ __forceinline__ Misc* misc(unsigned char* sm) { return reinterpret_cast<Misc*>(sm + OFF_MISC); }

// Waits for the MMAs committed so far; on a wait that runs out the CTA stops issuing tensor work
// (its results are then garbage and flagged) but keeps its place in every barrier.
__device__ __forceinline__ void mma_wait(unsigned char* sm, Counters* ctr) {
  Misc* ms = misc(sm);
  if (!ms->failed) {
    const bool ok = tc::mbar_wait_bounded(&ms->mbar, ms->phase, WAIT_LIMIT);
    __syncthreads();
    if (!ok) {
      if (threadIdx.x == 0) {
        ms->failed = 1;
        if (ctr) atomicAdd(&ctr->timeouts, 1ull);
      }
    }
    if (threadIdx.x == 0) ms->phase ^= 1u;
  }
  __syncthreads();
  tc::fence_after_sync();
}

// ---------------------------------------------------------------------------------- Gram
// D (TMEM, 128 x 128 fp32) = Z^T Z over rows [0, Mp) of the 64 columns cols[0..63] of the planes
// (Xr, Xi): Z column p < 64 is Re x_{cols[p]}, p >= 64 is Im x_{cols[p-64]}. Planes are
// column-major with leading dimension ld (a multiple of 4); Mp is a multiple of KC.
// Staging of one chunk of KC rows: core matrix (kc, pg) = (rows 4kc..4kc+3, Z columns 8pg..8pg+7)
// at byte ((kc * 16 + pg) * 8) * 16: LBO (along K) = 2048 B, SBO (along M/N) = 128 B.
__device__ void gram_pair(unsigned char* sm, const float* Xr, const float* Xi, int ld, int Mp, const int* cols,
                          Counters* ctr) {
  Misc* ms = misc(sm);
  float* st = reinterpret_cast<float*>(sm + OFF_STAGE);
  const uint32_t s_base = tc::smem_u32(sm + OFF_STAGE);
  constexpr uint32_t LBO = 2048, SBO = 128, LO = 16384;
  constexpr uint32_t ID = tc::idesc_tf32(128, 128);
  const int nchunks = Mp / KC;
  for (int c = 0; c < nchunks; ++c) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int e = threadIdx.x + THREADS * it;       // 1024 float4 of the chunk
      const int plo = e & 7, kc = (e >> 3) & 7, pg = e >> 6;
      const int p = pg * 8 + plo;
      const float* src = (p < P ? Xr + (size_t)cols[p] * ld : Xi + (size_t)cols[p - P] * ld) + c * KC + 4 * kc;
      // X changes between rounds (other CTAs of the cluster write it): read at L2, never through
      // the non-coherent read-only path or a possibly stale L1 line
      const float4 v = __ldcg(reinterpret_cast<const float4*>(src));
      float4 h, l;
      tc::split_tf32(v.x, h.x, l.x);
      tc::split_tf32(v.y, h.y, l.y);
      tc::split_tf32(v.z, h.z, l.z);
      tc::split_tf32(v.w, h.w, l.w);
      const int off = ((kc * 16 + pg) * 8 + plo) * 4;
      *reinterpret_cast<float4*>(st + off) = h;
      *reinterpret_cast<float4*>(st + LO / 4 + off) = l;
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0 && !ms->failed) {
      tc::fence_after_sync();
#pragma unroll
      for (int s = 0; s < KC / 8; ++s) {
        const uint32_t off = (uint32_t)s * 2 * LBO;
        const uint64_t ah = tc::smem_desc_kmajor(s_base + off, LBO, SBO);
        const uint64_t al = tc::smem_desc_kmajor(s_base + LO + off, LBO, SBO);
        const uint32_t acc0 = (c > 0 || s > 0) ? 1u : 0u;
        tc::mma_tf32(ms->tmem, ah, ah, ID, acc0);
        tc::mma_tf32(ms->tmem, ah, al, ID, 1u);
        tc::mma_tf32(ms->tmem, al, ah, ID, 1u);
      }
      tc::mma_commit(&ms->mbar);
    }
    mma_wait(sm, ctr);
  }
}

// H (64 x 64 complex, row-major with row stride HS in the staging area) from the Gram D = [[A, Bm], [Bm^T, C]]:
// Re H = A + C, Im H = Bm - Bm^T (H = Y^* Y). Warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows
// of D) and the column half w / 4.
__device__ void gram_to_h(unsigned char* sm) {
  Misc* ms = misc(sm);
  float2* H = reinterpret_cast<float2*>(sm + OFF_STAGE);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (w & 3) + lane;                  // row of D
  const int half = w >> 2;                              // D columns [64 half, 64 half + 64)
  const uint32_t ta = ms->tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(64 * half);
  // pass 1: rows < 64 write A (real part) or Bm (imaginary part); pass 2: rows >= 64 add C (real)
  // and subtract Bm^T (imaginary). 32 columns of D per TMEM load.
  for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
    for (int q0 = 0; q0 < 64; q0 += 32) {
      float v[32];
      tc::tmem_ld16(ta + q0, v);
      tc::tmem_ld16(ta + q0 + 16, v + 16);
      tc::tmem_ld_wait();
      if (pass == 0 && row < P) {
#pragma unroll
        for (int q = 0; q < 32; ++q) reinterpret_cast<float*>(H + row * HS + q0 + q)[half] = v[q];
      } else if (pass == 1 && row >= P) {
        const int r = row - P;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          float2* h = H + r * HS + q0 + q;
          if (half == 0) h->y -= v[q];      // D[64 + r][q] = (Bm^T)[r][q]
          else h->x += v[q];                // D[64 + r][64 + q] = C[r][q]
        }
      }
    }
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
}

// ---------------------------------------------------------------------------------- inner sweep
// Circle-method pair i of round t over 64 indices: (t, 63) for i = 0, else (c(t+i), c(t-i)),
// c(x) = x mod 63.
__device__ __forceinline__ void inner_pair(int t, int i, int& a, int& b) {
  if (i == 0) { a = t; b = P - 1; }
  else { a = (t + i) % (P - 1); b = (t - i + (P - 1)) % (P - 1); }
}

// One cyclic two-sided Jacobi sweep on H (staging area) accumulating Q (R1, fp32, starts as I).
// Returns the number of rotations (valid on thread 0..31 partial; summed by the caller).
__device__ int inner_sweep(unsigned char* sm, float tol2) {
  float2* H = reinterpret_cast<float2*>(sm + OFF_STAGE);
  float2* Q = reinterpret_cast<float2*>(sm + OFF_R1);
  float4* prm = reinterpret_cast<float4*>(sm + OFF_PRM);
  const uint16_t* tri = reinterpret_cast<const uint16_t*>(sm + OFF_TRI);
  Misc* ms = misc(sm);
  for (int e = threadIdx.x; e < P * P; e += THREADS)
    Q[e] = make_float2((e / P) == (e % P) ? 1.f : 0.f, 0.f);
  int nrot = 0;
  __syncthreads();
  for (int t = 0; t < P - 1; ++t) {
    if (threadIdx.x < 32) {
      int a, b;
      inner_pair(t, threadIdx.x, a, b);
      float al = H[a * HS + a].x, be = H[b * HS + b].x;
      const float2 g = H[a * HS + b];
      float gr = g.x, gi = g.y;
      const bool rot = pair_test(al, be, gr, gi, tol2);
      const float4 q = pair_params(al, be, gr, gi, rot);
      prm[threadIdx.x] = rot ? make_float4(q.x, q.y, q.z, 1.f) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (rot) { ++nrot; ms->rotated = 1; }
    }
    __syncthreads();
    // H <- J^* H J by 2x2 blocks (P <= P'), J = [[1 + cm1, es], [-conj(es), 1 + cm1]] per pair
    for (int e = threadIdx.x; e < 528; e += THREADS) {
      const int pp = tri[e] >> 8, qq = tri[e] & 0xff;    // pp <= qq
      const float4 jp = prm[pp], jq = prm[qq];
      if (jp.w == 0.f && jq.w == 0.f) continue;
      int a, b, c, d;
      inner_pair(t, pp, a, b);
      inner_pair(t, qq, c, d);
      float2 B00 = H[a * HS + c], B01 = H[a * HS + d], B10 = H[b * HS + c], B11 = H[b * HS + d];
      // T = B J_q: columns (c, d)
      float2 T00, T01, T10, T11;
      {
        const float cm = jq.x, er = jq.y, ei = jq.z;
        // t0 = b0 (1 + cm) - b1 conj(es); t1 = b0 es + b1 (1 + cm)
        T00 = make_float2(fmaf(cm, B00.x, B00.x) - (B01.x * er + B01.y * ei), fmaf(cm, B00.y, B00.y) - (B01.y * er - B01.x * ei));
        T01 = make_float2(fmaf(cm, B01.x, B01.x) + (B00.x * er - B00.y * ei), fmaf(cm, B01.y, B01.y) + (B00.x * ei + B00.y * er));
        T10 = make_float2(fmaf(cm, B10.x, B10.x) - (B11.x * er + B11.y * ei), fmaf(cm, B10.y, B10.y) - (B11.y * er - B11.x * ei));
        T11 = make_float2(fmaf(cm, B11.x, B11.x) + (B10.x * er - B10.y * ei), fmaf(cm, B11.y, B11.y) + (B10.x * ei + B10.y * er));
      }
      {
        const float cm = jp.x, er = jp.y, ei = jp.z;
        // row a' = (1 + cm) row_a - es row_b; row b' = conj(es) row_a + (1 + cm) row_b
        B00 = make_float2(fmaf(cm, T00.x, T00.x) - (T10.x * er - T10.y * ei), fmaf(cm, T00.y, T00.y) - (T10.x * ei + T10.y * er));
        B01 = make_float2(fmaf(cm, T01.x, T01.x) - (T11.x * er - T11.y * ei), fmaf(cm, T01.y, T01.y) - (T11.x * ei + T11.y * er));
        B10 = make_float2(fmaf(cm, T10.x, T10.x) + (T00.x * er + T00.y * ei), fmaf(cm, T10.y, T10.y) + (T00.y * er - T00.x * ei));
        B11 = make_float2(fmaf(cm, T11.x, T11.x) + (T01.x * er + T01.y * ei), fmaf(cm, T11.y, T11.y) + (T01.y * er - T01.x * ei));
      }
      H[a * HS + c] = B00;
      H[a * HS + d] = B01;
      H[b * HS + c] = B10;
      H[b * HS + d] = B11;
      if (pp != qq) {
        H[c * HS + a] = make_float2(B00.x, -B00.y);
        H[d * HS + a] = make_float2(B01.x, -B01.y);
        H[c * HS + b] = make_float2(B10.x, -B10.y);
        H[d * HS + b] = make_float2(B11.x, -B11.y);
      }
    }
    // Q <- Q J: every row x, every rotated pair
    for (int e = threadIdx.x; e < P * 32; e += THREADS) {
      const int x = e >> 5, i = e & 31;
      const float4 j = prm[i];
      if (j.w == 0.f) continue;
      int a, b;
      inner_pair(t, i, a, b);
      const float2 qa = Q[x * P + a], qb = Q[x * P + b];
      const float cm = j.x, er = j.y, ei = j.z;
      Q[x * P + a] = make_float2(fmaf(cm, qa.x, qa.x) - (qb.x * er + qb.y * ei), fmaf(cm, qa.y, qa.y) - (qb.y * er - qb.x * ei));
      Q[x * P + b] = make_float2(fmaf(cm, qb.x, qb.x) + (qa.x * er - qa.y * ei), fmaf(cm, qb.y, qb.y) + (qa.x * ei + qa.y * er));
    }
    __syncthreads();
  }
  return nrot;
}

// Q (R1, fp32 complex, Q[k][n] at k * 64 + n) -> the B operands of the update in R1: Re (Q - I)^T
// and Im Q^T (N = 64 output columns x K = 64), each split into TF32 hi and lo (16 KB each),
// K-major core matrices (kc, ng) at byte ((kc * 8 + ng) * 8) * 16: LBO = 1024 B, SBO = 128 B.
// Layout: [Re hi | Re lo | Im hi | Im lo]. The update forms Y (Q - I) on the tensor cores and adds
// Y exactly on the CUDA cores: the 3xTF32 error (a few fp32 units of each product) then scales
// with the rotation, which is small once the sweeps near convergence, instead of with Y.
__device__ void q_to_operands(unsigned char* sm) {
  float2* Q = reinterpret_cast<float2*>(sm + OFF_R1);
  float* R = reinterpret_cast<float*>(sm + OFF_R1);
  float2 q[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) q[j] = Q[threadIdx.x + THREADS * j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int e = threadIdx.x + THREADS * j;
    const int k = e / P, n = e % P;
    const int off = ((k / 4 * 8 + n / 8) * 8 + n % 8) * 4 + k % 4;
    float h, l;
    tc::split_tf32(k == n ? q[j].x - 1.f : q[j].x, h, l);
    R[off] = h;
    R[4096 + off] = l;
    tc::split_tf32(q[j].y, h, l);
    R[8192 + off] = h;
    R[12288 + off] = l;
  }
  tc::fence_proxy_async_smem();
  __syncthreads();
}

// ---------------------------------------------------------------------------------- update
// Rows [row0, row0 + 128) of the 64 columns cols[] of the planes (Pr, Pi) become Y Q = Y + Y (Q - I)
// (Y (Q - I) = [Re Y Re(Q - I) - Im Y Im Q, Re Y Im Q + Im Y Re(Q - I)] on the tensor cores, the
// R1 operands being those of Q - I), written to (Or, Oi) (may equal (Pr, Pi)).
// A chunk of KU = 16 columns of Y: Re and Im, each split hi/lo, 8 KB apiece, core matrix (kc, rg)
// = (columns 4kc..4kc+3, rows 8rg..8rg+7) at byte ((kc * 16 + rg) * 8) * 16: LBO = 2048, SBO = 128.
// TMEM columns [0, 64): Re Y', [64, 128): Im Y'.
__device__ void update_tile(unsigned char* sm, const float* Pr, const float* Pi, float* Or, float* Oi, int ld,
                            int row0, const int* cols, Counters* ctr) {
  Misc* ms = misc(sm);
  float* st = reinterpret_cast<float*>(sm + OFF_STAGE);
  const uint32_t s_base = tc::smem_u32(sm + OFF_STAGE);
  const uint32_t q_base = tc::smem_u32(sm + OFF_R1);
  constexpr uint32_t LBO = 2048, SBO = 128, QLBO = 1024, QSBO = 128;
  constexpr uint32_t ID = tc::idesc_tf32(128, 64);
  constexpr uint32_t ID_NEG = tc::idesc_tf32(128, 64, false, true);
  const int row = threadIdx.x & (RT - 1);
  const int kh = threadIdx.x >> 7;                       // this thread's column quads 2kh, 2kh + 1
  for (int u = 0; u < P / KU; ++u) {
#pragma unroll
    for (int qd = 0; qd < 2; ++qd) {
      const int kc = 2 * kh + qd;
      const int c0 = u * KU + 4 * kc;
      float4 vr, vi;
      const size_t r = (size_t)row0 + row;
      vr.x = __ldcg(Pr + (size_t)cols[c0] * ld + r);
      vr.y = __ldcg(Pr + (size_t)cols[c0 + 1] * ld + r);
      vr.z = __ldcg(Pr + (size_t)cols[c0 + 2] * ld + r);
      vr.w = __ldcg(Pr + (size_t)cols[c0 + 3] * ld + r);
      vi.x = __ldcg(Pi + (size_t)cols[c0] * ld + r);
      vi.y = __ldcg(Pi + (size_t)cols[c0 + 1] * ld + r);
      vi.z = __ldcg(Pi + (size_t)cols[c0 + 2] * ld + r);
      vi.w = __ldcg(Pi + (size_t)cols[c0 + 3] * ld + r);
      const int off = ((kc * 16 + (row >> 3)) * 8 + (row & 7)) * 4;
      float4 h, l;
      tc::split_tf32(vr.x, h.x, l.x);
      tc::split_tf32(vr.y, h.y, l.y);
      tc::split_tf32(vr.z, h.z, l.z);
      tc::split_tf32(vr.w, h.w, l.w);
      *reinterpret_cast<float4*>(st + off) = h;
      *reinterpret_cast<float4*>(st + 2048 + off) = l;
      tc::split_tf32(vi.x, h.x, l.x);
      tc::split_tf32(vi.y, h.y, l.y);
      tc::split_tf32(vi.z, h.z, l.z);
      tc::split_tf32(vi.w, h.w, l.w);
      *reinterpret_cast<float4*>(st + 4096 + off) = h;
      *reinterpret_cast<float4*>(st + 6144 + off) = l;
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0 && !ms->failed) {
      tc::fence_after_sync();
#pragma unroll
      for (int s = 0; s < KU / 8; ++s) {
        const uint32_t ao = (uint32_t)s * 2 * LBO;
        const uint64_t yrh = tc::smem_desc_kmajor(s_base + ao, LBO, SBO);
        const uint64_t yrl = tc::smem_desc_kmajor(s_base + 8192 + ao, LBO, SBO);
        const uint64_t yih = tc::smem_desc_kmajor(s_base + 16384 + ao, LBO, SBO);
        const uint64_t yil = tc::smem_desc_kmajor(s_base + 24576 + ao, LBO, SBO);
        const uint32_t qo = (uint32_t)((u * KU + 8 * s) / 4) * QLBO;
        const uint64_t qrh = tc::smem_desc_kmajor(q_base + qo, QLBO, QSBO);
        const uint64_t qrl = tc::smem_desc_kmajor(q_base + 16384 + qo, QLBO, QSBO);
        const uint64_t qih = tc::smem_desc_kmajor(q_base + 32768 + qo, QLBO, QSBO);
        const uint64_t qil = tc::smem_desc_kmajor(q_base + 49152 + qo, QLBO, QSBO);
        const uint32_t acc0 = (u > 0 || s > 0) ? 1u : 0u;
        const uint32_t dr = ms->tmem, di = ms->tmem + 64;
        // Re Y' = Re Y Re Q - Im Y Im Q
        tc::mma_tf32(dr, yrh, qrh, ID, acc0);
        tc::mma_tf32(dr, yrh, qrl, ID, 1u);
        tc::mma_tf32(dr, yrl, qrh, ID, 1u);
        tc::mma_tf32(dr, yih, qih, ID_NEG, 1u);
        tc::mma_tf32(dr, yih, qil, ID_NEG, 1u);
        tc::mma_tf32(dr, yil, qih, ID_NEG, 1u);
        // Im Y' = Re Y Im Q + Im Y Re Q
        tc::mma_tf32(di, yrh, qih, ID, acc0);
        tc::mma_tf32(di, yrh, qil, ID, 1u);
        tc::mma_tf32(di, yrl, qih, ID, 1u);
        tc::mma_tf32(di, yih, qrh, ID, 1u);
        tc::mma_tf32(di, yih, qrl, ID, 1u);
        tc::mma_tf32(di, yil, qrh, ID, 1u);
      }
      tc::mma_commit(&ms->mbar);
    }
    mma_wait(sm, ctr);
  }
  // epilogue: warps 0-3 write Re Y' (TMEM columns 0..63), warps 4-7 Im Y' (64..127)
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int orow = 32 * (w & 3) + lane;
  const uint32_t ta = ms->tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(64 * (w >> 2));
  float* O = (w >> 2) ? Oi : Or;
  const size_t r = (size_t)row0 + orow;
#pragma unroll
  for (int q0 = 0; q0 < 64; q0 += 32) {
    float v[32];
    tc::tmem_ld16(ta + q0, v);
    tc::tmem_ld16(ta + q0 + 16, v + 16);
    tc::tmem_ld_wait();
    const float* Y = (w >> 2) ? Pi : Pr;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const size_t e = (size_t)cols[q0 + q] * ld + r;
      O[e] = __ldcg(Y + e) + v[q];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
}

// ---------------------------------------------------------------------------------- set-up
__device__ void cta_setup(unsigned char* sm) {
  Misc* ms = misc(sm);
  uint16_t* tri = reinterpret_cast<uint16_t*>(sm + OFF_TRI);
  for (int e = threadIdx.x; e < 32 * 32; e += THREADS) {
    const int p = e >> 5, q = e & 31;
    if (p <= q) tri[q * (q + 1) / 2 + p] = (uint16_t)((p << 8) | q);
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(&ms->mbar, 1);
    tc::fence_mbar_init();
    ms->phase = 0;
    ms->failed = 0;
    ms->rotated = 0;
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(&ms->tmem, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

__device__ void cta_teardown(unsigned char* sm) {
  Misc* ms = misc(sm);
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(ms->tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------------- symbol kernel
// Block pair of position `pos` at round t of the circle method over nb blocks: (t, nb - 1) for
// position 0, else (c(t + pos), c(t - pos)), c(x) = x mod (nb - 1).
__device__ __forceinline__ void outer_pair(int t, int pos, int nb, int& I, int& J) {
  const int Cn = nb - 1;
  if (pos == 0) { I = t % Cn; J = nb - 1; }
  else { I = (t + pos) % Cn; J = (t - pos + Cn) % Cn; }
}

}  // namespace bj

// One symbol per thread-block cluster of CS = Np / 64 CTAs (see the file comment). Per symbol:
// assembly of X = A_k (or A_k^*) into the cluster's workspace slot, W = I; sweeps of nb - 1 rounds;
// then sigma, ranks and the normalised factors written to the layer's outputs.
template <int CS, bool VEC>
__global__ void __launch_bounds__(bj::THREADS, 2) bj_kernel(const __grid_constant__ BJLaunch A) {
  using namespace bj;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ int scols[P];
  __shared__ float sinv[2][P];          // 1/|x_c| (0 for a negligible column), 1/|w_c| of this CTA's columns
  __shared__ int srank[P];
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const int slot = blockIdx.x / CS;
  const LayerArgs& La = A.L;
  Counters* ctr = A.counters;
  const int Mp = A.Mp, Np = A.Np, ldx = A.ldx, ldw = A.ldw;
  const int M = La.M, N = La.N;
  const int nb = Np / B;
  float* Xr = A.ws + (size_t)slot * A.slot_floats;
  float* Xi = Xr + (size_t)Np * ldx;
  float* Wr = Xi + (size_t)Np * ldx;
  float* Wi = Wr + (size_t)Np * ldw;
  float* sg = VEC ? Wi + (size_t)Np * ldw : Wr;   // sigma of every column of the symbol
  float2* phs = reinterpret_cast<float2*>(sm + OFF_PHS);
  Misc* ms = misc(sm);
  cta_setup(sm);
  cl.sync();   // every CTA of the cluster has started before rank 0 writes into their shared memory
  unsigned int* queue = &ctr->queue[A.queue_slot];
  const int c_beg = crank * (Np / CS), c_end = c_beg + Np / CS;   // this CTA's 64 columns

  for (;;) {
    if (crank == 0 && threadIdx.x == 0) {
      const int it = (int)atomicAdd(queue, 1u);
      for (int r = 0; r < CS; ++r) *cl.map_shared_rank(&ms->item, r) = it;
      ms->vote[0] = 0;
      ms->vote[1] = 0;
    }
    cl.sync();
    const int h = ms->item;
    if (h >= A.total_items) break;
    const int f = La.half[h];
    const int jj = f / La.m, ll = f - jj * La.m;
    const int kk = La.kh * La.kw;
    for (int t = threadIdx.x; t < kk; t += THREADS) phs[t] = tap_phase(La, jj, ll, t / La.kw, t % La.kw);
    __syncthreads();
    // ---- X = the symbol (assembled from the taps), W = I; padding rows and columns are zero
    for (int c = c_beg; c < c_end; ++c) {
      for (int row = threadIdx.x; row < Mp; row += THREADS) {
        const float2 v = x_entry<true>(La, h, row, c, phs);
        Xr[(size_t)c * ldx + row] = v.x;
        Xi[(size_t)c * ldx + row] = v.y;
      }
      if constexpr (VEC) {
        for (int row = threadIdx.x; row < Np; row += THREADS) {
          Wr[(size_t)c * ldw + row] = (row == c && c < N) ? 1.f : 0.f;
          Wi[(size_t)c * ldw + row] = 0.f;
        }
      }
    }
    __threadfence();
    cl.sync();
    // ---- sweeps
    int sweeps = 0, nrot = 0;
    bool converged = false;
    for (;;) {
      int rotated_sweep = 0;
      for (int t = 0; t < nb - 1; ++t) {
        int I, J;
        outer_pair(t, crank, nb, I, J);
        if (threadIdx.x < P) scols[threadIdx.x] = threadIdx.x < B ? I * B + threadIdx.x : J * B + threadIdx.x - B;
        if (threadIdx.x == 0) ms->rotated = 0;
        __syncthreads();
        gram_pair(sm, Xr, Xi, ldx, Mp, scols, ctr);
        gram_to_h(sm);
        nrot += inner_sweep(sm, La.tol2);
        if (ms->rotated) {
          rotated_sweep = 1;
          q_to_operands(sm);
          for (int r0 = 0; r0 < Mp; r0 += RT) update_tile(sm, Xr, Xi, Xr, Xi, ldx, r0, scols, ctr);
          if constexpr (VEC)
            for (int r0 = 0; r0 < Np; r0 += RT) update_tile(sm, Wr, Wi, Wr, Wi, ldw, r0, scols, ctr);
        }
        __threadfence();
        cl.sync();
      }
      ++sweeps;
      const int q = sweeps & 1;
      if (threadIdx.x == 0 && rotated_sweep) atomicOr(cl.map_shared_rank(&ms->vote[q], 0), 1);
      cl.sync();
      const int any = *cl.map_shared_rank(&ms->vote[q], 0);
      if (crank == 0 && threadIdx.x == 0) ms->vote[q ^ 1] = 0;    // the slot of the next sweep
      if (!any) { converged = true; break; }
      if (sweeps >= A.max_sweeps) break;
    }
    if (crank == 0 && threadIdx.x == 0) {
      atomicAdd(&ctr->sweeps, (unsigned long long)sweeps);
      if (!converged) atomicAdd(&ctr->unconverged, 1ull);
    }
    if (threadIdx.x < 32 && nrot) atomicAdd(&ctr->rotations, (unsigned long long)nrot);
    // ---- sigma_c = |x_c| / |w_c| for this CTA's columns (x_c = A w_c to rounding)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int cl_ = w; cl_ < P; cl_ += THREADS / 32) {
      const int c = c_beg + cl_;
      float xn = 0.f, wn = 0.f;
      for (int row = lane; row < Mp; row += 32) {
        const float a = __ldcg(Xr + (size_t)c * ldx + row), b = __ldcg(Xi + (size_t)c * ldx + row);
        xn = fmaf(a, a, fmaf(b, b, xn));
      }
      if constexpr (VEC) {
        for (int row = lane; row < Np; row += 32) {
          const float a = __ldcg(Wr + (size_t)c * ldw + row), b = __ldcg(Wi + (size_t)c * ldw + row);
          wn = fmaf(a, a, fmaf(b, b, wn));
        }
      } else {
        wn = 1.f;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        xn += __shfl_xor_sync(0xffffffffu, xn, o);
        wn += __shfl_xor_sync(0xffffffffu, wn, o);
      }
      if constexpr (!VEC) wn = 1.f;   // values only: W is not tracked, |w_c| = 1
      const float ixn = xn > 0x1p-100f ? rsqrt_nr(xn) : 0.f;   // the sweeps' zero-column bound
      const float iwn = wn > 0.f ? rsqrt_nr(wn) : 0.f;
      if (lane == 0) {
        sg[c] = c < N ? xn * ixn * iwn : -1.f;
        sinv[0][cl_] = ixn;
        sinv[1][cl_] = iwn;
      }
    }
    __threadfence();
    cl.sync();
    // ---- ranks (descending sigma, ties by column index) and sigma
    if (threadIdx.x < P) {
      const int c = c_beg + threadIdx.x;
      const float sc = __ldcg(sg + c);
      int rank = 0;
      bool finite = true;
      float smax = 0.f;
      for (int q2 = 0; q2 < N; ++q2) {
        const float v = __ldcg(sg + q2);
        finite = finite && isfinite(v);
        smax = fmaxf(smax, v);
        rank += (v > sc) || (v == sc && q2 < c);
      }
      srank[threadIdx.x] = c < N ? rank : -1;
      // a column far below sigma_max carries no direction: written as zero, completed afterwards
      if (!(sc > 1e-12f * smax)) sinv[0][threadIdx.x] = 0.f;
      if (c < N) {
        float* srow = La.sigma + (size_t)(A.half_output ? h : f) * La.r;
        srow[rank] = sc;
        if (!A.half_output) {
          const int fc = ((La.n - jj) % La.n) * La.m + (La.m - ll) % La.m;
          if (fc != f) La.sigma[(size_t)fc * La.r + rank] = sc;
        }
      }
      if (threadIdx.x == 0 && crank == 0 && !finite) atomicAdd(&ctr->nonfinite, 1ull);
    }
    __syncthreads();
    if constexpr (VEC) {
      float2* Xo = (La.wide ? La.V : La.U) + (size_t)h * M * N;
      float2* Wo = (La.wide ? La.U : La.V) + (size_t)h * N * N;
      for (int cl_ = 0; cl_ < P; ++cl_) {
        const int c = c_beg + cl_, rk = srank[cl_];
        if (rk < 0) continue;
        const float ix = sinv[0][cl_], iw = sinv[1][cl_];
        for (int row = threadIdx.x; row < M; row += THREADS)
          Xo[(size_t)row * N + rk] = make_float2(__ldcg(Xr + (size_t)c * ldx + row) * ix,
                                                 __ldcg(Xi + (size_t)c * ldx + row) * ix);
        for (int row = threadIdx.x; row < N; row += THREADS)
          Wo[(size_t)row * N + rk] = make_float2(__ldcg(Wr + (size_t)c * ldw + row) * iw,
                                                 __ldcg(Wi + (size_t)c * ldw + row) * iw);
      }
    }
    __threadfence();
    cl.sync();   // the slot is reused by the cluster's next symbol
  }
  cl.sync();
  cta_teardown(sm);
}

template <int CS, bool VEC>
static cudaError_t bj_config(int sms, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int* max_clusters) {
  cudaError_t e = cudaFuncSetAttribute(bj_kernel<CS, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bj::SMEM);
  if (e != cudaSuccess) return e;
  cfg = {};
  cfg.gridDim = dim3((unsigned)CS, 1, 1);
  cfg.blockDim = dim3(bj::THREADS, 1, 1);
  cfg.dynamicSmemBytes = bj::SMEM;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (max_clusters) {
    int nc = 0;
    e = cudaOccupancyMaxActiveClusters(&nc, bj_kernel<CS, VEC>, &cfg);
    if (e != cudaSuccess) return e;
    // two CTAs per SM at most: each holds TMEM_COLS of the SM's 512 tensor-memory columns
    *max_clusters = std::min(nc, 2 * sms / CS);
  }
  return cudaSuccess;
}

template <int CS, bool VEC>
static cudaError_t bj_launch_t(const BJLaunch& A, int clusters, cudaStream_t s) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e = bj_config<CS, VEC>(0, cfg, attr, nullptr);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3((unsigned)(clusters * CS), 1, 1);
  cfg.stream = s;
  return cudaLaunchKernelEx(&cfg, bj_kernel<CS, VEC>, A);
}

bool bj_supported(int M, int N) { return M >= 1 && N >= 1 && M <= 512 && N <= 512; }
void bj_dims(int M, int N, int* Mp, int* Np) {
  *Mp = (M + bj::RT - 1) / bj::RT * bj::RT;
  *Np = (N + 127) / 128 * 128;
}

cudaError_t bj_max_clusters(int M, int N, bool vec, int sms, int* clusters) {
  int Mp, Np;
  bj_dims(M, N, &Mp, &Np);
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  switch (Np / 64) {
    case 2: return vec ? bj_config<2, true>(sms, cfg, attr, clusters) : bj_config<2, false>(sms, cfg, attr, clusters);
    case 4: return vec ? bj_config<4, true>(sms, cfg, attr, clusters) : bj_config<4, false>(sms, cfg, attr, clusters);
    case 6: return vec ? bj_config<6, true>(sms, cfg, attr, clusters) : bj_config<6, false>(sms, cfg, attr, clusters);
    case 8: return vec ? bj_config<8, true>(sms, cfg, attr, clusters) : bj_config<8, false>(sms, cfg, attr, clusters);
  }
  return cudaErrorInvalidValue;
}

size_t bj_slot_floats(int M, int N, bool vec) {
  int Mp, Np;
  bj_dims(M, N, &Mp, &Np);
  return (size_t)2 * Np * Mp + (vec ? (size_t)2 * Np * Np : 0) + (size_t)Np;
}

cudaError_t launch_bj(const BJLaunch& A, int clusters, bool vec, cudaStream_t s) {
  switch (A.Np / 64) {
    case 2: return vec ? bj_launch_t<2, true>(A, clusters, s) : bj_launch_t<2, false>(A, clusters, s);
    case 4: return vec ? bj_launch_t<4, true>(A, clusters, s) : bj_launch_t<4, false>(A, clusters, s);
    case 6: return vec ? bj_launch_t<6, true>(A, clusters, s) : bj_launch_t<6, false>(A, clusters, s);
    case 8: return vec ? bj_launch_t<8, true>(A, clusters, s) : bj_launch_t<8, false>(A, clusters, s);
  }
  return cudaErrorInvalidValue;
}

// ================================================================================== debug kernels
// One CTA: the Gram of one block pair (the tensor-core contraction of the route), written out.
__global__ void __launch_bounds__(bj::THREADS, 1)
bj_gram_test_kernel(const float* Xr, const float* Xi, int ld, int Mp, const int* cols, float* D, Counters* ctr) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ int scol[bj::P];
  if (threadIdx.x < bj::P) scol[threadIdx.x] = cols[threadIdx.x];
  bj::cta_setup(sm);
  bj::gram_pair(sm, Xr, Xi, ld, Mp, scol, ctr);
  bj::gram_to_h(sm);
  const float2* H = reinterpret_cast<const float2*>(sm + bj::OFF_STAGE);
  for (int e = threadIdx.x; e < bj::P * bj::P; e += bj::THREADS) {
    const float2 v = H[(e / bj::P) * bj::HS + e % bj::P];
    D[2 * e] = v.x;
    D[2 * e + 1] = v.y;
  }
  bj::cta_teardown(sm);
}

// One CTA: Y Q for the 64 columns cols[] over rows [0, rows) (rows a multiple of 128), Q complex
// [64][64] row-major, written to (Or, Oi).
__global__ void __launch_bounds__(bj::THREADS, 1)
bj_update_test_kernel(const float* Pr, const float* Pi, float* Or, float* Oi, int ld, int rows, const int* cols,
                      const float2* Qin, Counters* ctr) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ int scol[bj::P];
  if (threadIdx.x < bj::P) scol[threadIdx.x] = cols[threadIdx.x];
  bj::cta_setup(sm);
  float2* Q = reinterpret_cast<float2*>(sm + bj::OFF_R1);
  for (int e = threadIdx.x; e < bj::P * bj::P; e += bj::THREADS) Q[e] = Qin[e];
  __syncthreads();
  bj::q_to_operands(sm);
  for (int r0 = 0; r0 < rows; r0 += bj::RT) bj::update_tile(sm, Pr, Pi, Or, Oi, ld, r0, scol, ctr);
  bj::cta_teardown(sm);
}

cudaError_t launch_bj_gram_test(const float* Xr, const float* Xi, int ld, int Mp, const int* cols, float* D,
                                Counters* ctr, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(bj_gram_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bj::SMEM);
  if (e != cudaSuccess) return e;
  bj_gram_test_kernel<<<1, bj::THREADS, bj::SMEM, s>>>(Xr, Xi, ld, Mp, cols, D, ctr);
  return cudaGetLastError();
}

cudaError_t launch_bj_update_test(const float* Pr, const float* Pi, float* Or, float* Oi, int ld, int rows,
                                  const int* cols, const float2* Q, Counters* ctr, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(bj_update_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bj::SMEM);
  if (e != cudaSuccess) return e;
  bj_update_test_kernel<<<1, bj::THREADS, bj::SMEM, s>>>(Pr, Pi, Or, Oi, ld, rows, cols, Q, ctr);
  return cudaGetLastError();
}

}  // namespace lfa

// ================================================================================== debug hooks
extern "C" {

// The tensor-core Gram of one block pair: H = Y^* Y for the 64 columns cols[] (device int32) of
// the column-major planes (Xr, Xi) with leading dimension ld over rows [0, Mp) (Mp a multiple of
// 32, ld a multiple of 4); H written to D as complex64 [64][64]. Returns 0, or the CUDA error.
int32_t lfa_debug_tc_gram(const float* Xr, const float* Xi, int32_t ld, int32_t Mp, const int32_t* cols, float* D,
                          void* stream) {
  if (!Xr || !Xi || !cols || !D || ld < Mp || (ld & 3) || Mp < 32 || (Mp & 31)) return -1;
  const cudaError_t e = lfa::launch_bj_gram_test(Xr, Xi, ld, Mp, cols, D, nullptr, static_cast<cudaStream_t>(stream));
  return (int32_t)e;
}

// The tensor-core update of one block pair: rows [0, rows) of the columns cols[] of (Pr, Pi)
// times Q (device complex64 [64][64] row-major), written to (Or, Oi) in the same layout. rows a
// multiple of 128. Returns 0, or the CUDA error.
int32_t lfa_debug_tc_update(const float* Pr, const float* Pi, float* Or, float* Oi, int32_t ld, int32_t rows,
                            const int32_t* cols, const float* Q, void* stream) {
  if (!Pr || !Pi || !Or || !Oi || !cols || !Q || ld < rows || rows < 128 || (rows & 127)) return -1;
  const cudaError_t e = lfa::launch_bj_update_test(Pr, Pi, Or, Oi, ld, rows, cols, reinterpret_cast<const float2*>(Q),
                                                   nullptr, static_cast<cudaStream_t>(stream));
  return (int32_t)e;
}

}  // extern "C"
