// Blocked one-sided Jacobi SVD of large LFA symbols on the tcgen05 tensor cores (arXiv 2506.05617,
// Sec. III: the SVD A_k = U_k S_k V_k^* of each symbol, Algorithm 1 line 5), for symbols whose
// element-wise Jacobi is far from the FP32 roofline (c >= 128).
//
// Method (Hestenes' one-sided Jacobi, applied to blocks of columns): X = A_k (or A_k^* for wide
// symbols) has its N columns split into nb blocks of 32. A sweep visits every pair of blocks
// (I, J) once, in the circle-method order over blocks (nb / 2 disjoint pairs per round). For a
// pair, Y = [X_I, X_J] (M x 64) gives the Hermitian Gram matrix H = Y^* Y (64 x 64); one
// two-sided Jacobi sweep over H (rounds of 32 disjoint 2x2 rotations, each rotation chosen only
// when |h_pq| > tol sqrt(h_pp h_qq), the one-sided test: all 63 rounds of the circle method in
// the first round of an outer sweep, the 32 rounds of the pairs across the two blocks otherwise)
// accumulates the unitary Q, and Y and the matching columns of W (the accumulated right factor,
// W = I initially) are replaced by Y Q and W Q. Because X = A W holds for any right factor, x_c = A w_c stays exact to
// rounding; sweeps repeat until no pair of a sweep rotates. Then sigma_c = |x_c| / |w_c|, the X
// columns normalised give U (V for wide symbols) and the W columns V (U).
//
// GB300 mapping:
//  * The two dense contractions of a block pair run on the tensor cores with TF32 operands
//    split 3 ways (hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor memory), which keeps
//    FP32 accuracy: the Gram in real form, Z^T Z with Z = [Re Y, Im Y] (M x 128, one
//    128 x 128 MMA tile, K = M), and the update Y (Q - I) as Re Y B and Im Y B with
//    B = [Re(Q - I) | Im Q] (M = 128-row tiles, N = 128, K = 64), combined and added to Y on the
//    CUDA cores. Operands are staged by the CTA's threads (which split fp32 into TF32 pairs) in
//    K-major core-matrix layout; one thread issues the MMAs and an mbarrier reports their
//    completion.
//  * The inner 64 x 64 problem runs on the CUDA cores from shared memory.
//  * One CTA of 256 threads works on one symbol (X and W, 4 MB at 512 x 512, in its workspace
//    slot), taking the block pairs of each round in turn; CTAs pull symbols from an atomic work
//    queue. Two CTAs share an SM (each ~100 KB of shared memory and half of the tensor memory):
//    a block pair's phases are chains of barriers and dependent loads, and the other CTA's
//    symbol fills those gaps. (One 512-thread CTA per SM was measured first: 2.82 s for the
//    512 -> 512 layer on 64 x 64; one thread-block cluster per symbol, one block pair per CTA and
//    round, before that: the rounds waited on the cluster barrier.)
#include <algorithm>

#include "jacobi.cuh"
#include "lfa_internal.cuh"
#include "tc_ptx.cuh"

namespace lfa {


namespace bj {

constexpr int B = 32;            // columns per block
constexpr int P = 2 * B;         // columns of a block pair
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 2;   // two symbols per SM: one CTA's barriers and loads hide the other's
constexpr int MAX_REGS = 120;    // registers per thread: two CTAs of 256 threads fit the register file
                                 // (at 128 the occupancy calculator admits one)
constexpr int KC = 32;           // rows of X per Gram chunk (K of the Gram)
constexpr int RT = 128;          // rows of X (or W) per update tile (M of the update)
constexpr int KU = 8;            // columns of Y per update chunk (K of one MMA)
constexpr uint32_t TMEM_COLS = 256;   // Gram D (128 columns), or two update accumulators
constexpr uint32_t WAIT_LIMIT = 1u << 22;
constexpr int HS = P + 1;        // row stride of H (float2): a column of H spreads over the banks

// Shared memory (bytes). Two CTAs share an SM, so each phase of a block pair reuses one 97 KB
// region (the phases of one CTA never overlap):
//  Gram:          chunk buffer 0 [0, 32K) | chunk buffer 1 [32K, 64K)   (TF32 hi | lo, 16 KB each)
//  inner sweep:   Q in fp32 [0, 32K) | H (64 x 65 float2) [32K, 32K + 33280)
//  update:        Q operands [0, 64K) | two update chunk buffers [65K, 97K) (16 KB each)
constexpr int OFF_STAGE = 0;               // Gram buffer 0, Q, Q operands
constexpr int OFF_R1 = 32768;              // Gram buffer 1, H
constexpr int OFF_UPD = 66560;             // update chunk buffers (after H)
constexpr int REGION_BYTES = OFF_UPD + 32768;
constexpr int OFF_PRM = REGION_BYTES;                // float4 [32] rotation parameters of a round
constexpr int OFF_PAB = OFF_PRM + 32 * 16;           // int32 [2][32] the round's pairs (a, b)
constexpr int OFF_TRI = OFF_PAB + 256;               // uint16 [528] pair-block (P, P') table
constexpr int OFF_PHS = OFF_TRI + 1088;              // float2 [256] phases of the symbol
constexpr int OFF_MISC = OFF_PHS + kMaxTaps * 8;     // mbarriers, tmem base, flags
constexpr int SMEM = OFF_MISC + 64;
static_assert(OFF_R1 + P * HS * 8 <= OFF_UPD, "H ends before the update buffers");
static_assert(P * P * 8 <= OFF_R1, "Q (fp32) ends before H");
static_assert(2 * KC * 2 * P * 4 <= OFF_R1 && 4 * P * P * 4 <= OFF_UPD && OFF_UPD + 2 * 4 * RT * KU * 4 <= REGION_BYTES,
              "Gram buffers, Q operands and update buffers fit their places");
static_assert(OFF_R1 % 1024 == 0 && OFF_UPD % 1024 == 0 && OFF_PRM % 16 == 0 && OFF_PHS % 16 == 0 &&
              OFF_MISC % 16 == 0, "alignment");
static_assert(CTAS_PER_SM * (SMEM + 2048) <= 233472, "two CTAs per SM");

constexpr int MB_TILE = 2;       // mbarrier of a finished update tile
struct Misc {
  uint64_t mbar[3];     // [0], [1]: MMA completion, one per operand buffer; [MB_TILE]: an update tile
  uint32_t tmem;        // TMEM base column address
  int32_t rotated;      // the block pair rotated in its inner sweep
  int32_t failed;       // a bounded wait ran out: no further tensor work in this CTA
  int32_t item;         // work item
  int32_t any;          // some pair of the block pair passes the rotation test
  int32_t warm;         // the symbol starts from its predecessor's V
  int32_t pad[4];
};
static_assert(sizeof(Misc) <= 64, "misc block");

__device__ __forceinline__ Misc* misc(unsigned char* sm) { return reinterpret_cast<Misc*>(sm + OFF_MISC); }

// Waits until the MMAs committed to mbarrier b have completed. Every thread tracks the two phase
// parities in `ph` (all threads run the same sequence of waits). A wait that runs out marks the CTA
// failed: it issues no further tensor work and skips later waits (its results are garbage and
// counted as a timeout) but keeps its place in every barrier.
__device__ __forceinline__ void wait_buf(unsigned char* sm, Counters* ctr, int b, uint32_t& ph) {
  Misc* ms = misc(sm);
  if (!*reinterpret_cast<volatile int32_t*>(&ms->failed)) {
    if (!tc::mbar_wait_bounded(&ms->mbar[b], (ph >> b) & 1u, WAIT_LIMIT))
      if (atomicExch(&ms->failed, 1) == 0 && ctr) atomicAdd(&ctr->timeouts, 1ull);
  }
  ph ^= 1u << b;
  tc::fence_after_sync();
}

// ---------------------------------------------------------------------------------- Gram
// D (TMEM columns [0, 128), 128 x 128 fp32) = Z^T Z over rows [0, Mp) of the 64 columns cols[] of
// the planes (Xr, Xi): Z column p < 64 is Re x_{cols[p]}, p >= 64 is Im x_{cols[p-64]}. Planes are
// column-major with leading dimension ld (a multiple of 4); Mp is a multiple of KC.
// A chunk of KC = 32 rows is staged as TF32 hi | lo (16 KB each), core matrix (kc, pg) = (rows
// 4kc..4kc+3, Z columns 8pg..8pg+7) at byte ((kc * 16 + pg) * 8) * 16: LBO (along K) = 2048 B, SBO
// (along M/N) = 128 B.
// Two chunk buffers alternate; the next two chunks are in flight (asynchronous copies into raw
// buffers) while the tensor core works on the current one.
__device__ void gram_pair(unsigned char* sm, const float* Xr, const float* Xi, int ld, int Mp, const int* cols,
                          Counters* ctr, uint32_t& ph) {
  Misc* ms = misc(sm);
  constexpr uint32_t LBO = 2048, SBO = 128, LO = KC * 2 * P * 4;
  constexpr uint32_t ID = tc::idesc_tf32(128, 128);
  constexpr int RAW = KC * 2 * P * 4;               // bytes of one raw chunk (fp32, staged layout)
  static_assert(OFF_UPD + 2 * RAW <= REGION_BYTES, "two raw chunks fit the update buffers' place");
  const uint32_t base0 = tc::smem_u32(sm + OFF_STAGE), base1 = tc::smem_u32(sm + OFF_R1);
  constexpr int NIT = KC * 2 * P / 4 / THREADS;   // float4 per thread and chunk
  const float* src[NIT];
  int off[NIT];
#pragma unroll
  for (int it = 0; it < NIT; ++it) {
    const int e = threadIdx.x + THREADS * it;       // KC * 128 / 4 float4 per chunk
    const int plo = e & 7, kc = (e >> 3) & (KC / 4 - 1), pg = e / (8 * KC / 4);
    const int p = pg * 8 + plo;
    src[it] = (p < P ? Xr + (size_t)cols[p] * ld : Xi + (size_t)cols[p - P] * ld) + 4 * kc;
    off[it] = ((kc * 16 + pg) * 8 + plo) * 4;
  }
  // Raw chunks arrive by asynchronous copies (at L2: X is rewritten by the update epilogues) into two
  // raw buffers in the update buffers' place, two chunks ahead; each thread converts the float4s it
  // copied itself, so its own wait_group is the only synchronisation the raw data needs.
  float* raw = reinterpret_cast<float*>(sm + OFF_UPD);
  const int n = Mp / KC;
  auto fetch = [&](int c) {
    float* r = raw + (c & 1) * (RAW / 4);
#pragma unroll
    for (int it = 0; it < NIT; ++it) tc::cp_async16(r + off[it], src[it] + c * KC);
  };
  fetch(0);
  tc::cp_async_commit();
  if (n > 1) fetch(1);
  tc::cp_async_commit();
  for (int c = 0; c < n; ++c) {
    const int b = c & 1;
    float* st = reinterpret_cast<float*>(sm + (b ? OFF_R1 : OFF_STAGE));
    tc::cp_async_wait<1>();                         // chunk c has arrived (c + 1 may be in flight)
    const float* r = raw + b * (RAW / 4);
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const float4 v = *reinterpret_cast<const float4*>(r + off[it]);
      float4 h, l;
      tc::split_tf32(v.x, h.x, l.x);
      tc::split_tf32(v.y, h.y, l.y);
      tc::split_tf32(v.z, h.z, l.z);
      tc::split_tf32(v.w, h.w, l.w);
      *reinterpret_cast<float4*>(st + off[it]) = h;
      *reinterpret_cast<float4*>(st + LO / 4 + off[it]) = l;
    }
    if (c + 2 < n) fetch(c + 2);                    // into the raw buffer this thread just read
    tc::cp_async_commit();
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0 && !ms->failed) {
      tc::fence_after_sync();
#pragma unroll
      for (int s = 0; s < KC / 8; ++s) {
        const uint32_t o = (uint32_t)s * 2 * LBO;
        const uint32_t bb = b ? base1 : base0;
        const uint64_t ah = tc::smem_desc_kmajor(bb + o, LBO, SBO);
        const uint64_t al = tc::smem_desc_kmajor(bb + LO + o, LBO, SBO);
        const uint32_t acc0 = (c > 0 || s > 0) ? 1u : 0u;
        tc::mma_tf32(ms->tmem, ah, ah, ID, acc0);
        tc::mma_tf32(ms->tmem, ah, al, ID, 1u);
        tc::mma_tf32(ms->tmem, al, ah, ID, 1u);
      }
      tc::mma_commit(&ms->mbar[b]);
    }
    if (c >= 1) wait_buf(sm, ctr, (c - 1) & 1, ph);   // chunk c - 1 done: its buffer is free for c + 1
  }
  tc::cp_async_wait<0>();
  wait_buf(sm, ctr, (n - 1) & 1, ph);
}

// H (64 x 64 complex, row-major with row stride HS at OFF_R1) from the Gram
// D = [[A, Bm], [Bm^T, C]]: Re H = A + C, Im H = Bm - Bm^T (H = Y^* Y). Warp w reads TMEM lanes
// 32 (w % 4) .. + 31 (rows of D) and, in turn, the column groups g = w / 4, w / 4 + THREADS / 128, ...
// of D (group g: columns 64 (g / 2) + 32 (g % 2) .. + 31). Then every pair (p, q) the inner sweep
// visits (all pairs when `full`, else the pairs across the two blocks) is tested with the rotation
// rule: misc->any = 0 means the inner sweep would not rotate at all.
__device__ void gram_to_h(unsigned char* sm, float tol2, bool full) {
  Misc* ms = misc(sm);
  float2* H = reinterpret_cast<float2*>(sm + OFF_R1);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (w & 3) + lane;                  // row of D
  if (threadIdx.x == 0) ms->any = 0;
  // pass 1: rows < 64 write A (real part) or Bm (imaginary part); pass 2: rows >= 64 add C (real)
  // and subtract Bm^T (imaginary). 32 columns of D per TMEM load.
  for (int pass = 0; pass < 2; ++pass) {
    for (int g = w >> 2; g < 4; g += THREADS / 128) {
      const int half = g >> 1;                          // D columns [64 half, 64 half + 64) ...
      const int q0 = (g & 1) * 32;                      // ... of which [q0, q0 + 32)
      const uint32_t ta = ms->tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(64 * half + q0);
      float v[32];
      tc::tmem_ld16(ta, v);
      tc::tmem_ld16(ta + 16, v + 16);
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
  // the rotation test on the pairs of the initial H that the inner sweep visits
  bool any = false;
  for (int e = threadIdx.x; e < P * P; e += THREADS) {
    const int p = e >> 6, q = e & 63;
    if (p >= q || (!full && q < B) || (!full && p >= B)) continue;
    float al = H[p * HS + p].x, be = H[q * HS + q].x;
    const float2 g = H[p * HS + q];
    float gr = g.x, gi = g.y;
    any = any || pair_test(al, be, gr, gi, tol2);
  }
  if (any) ms->any = 1;
  __syncthreads();
}

// ---------------------------------------------------------------------------------- inner sweep
// Pair i of round t of the inner sweep over the 64 columns of a block pair. A full sweep (63 rounds)
// takes the circle method over all 64 indices: (t, 63) for i = 0, else (c(t+i), c(t-i)),
// c(x) = x mod 63. A cross sweep (32 rounds) visits only the 32 x 32 pairs across the two blocks:
// (i, 32 + (i + t) mod 32). The outer sweep gives every block pair of its first round a full inner
// sweep (each block occurs once in that round, so every pair inside a block is visited once per
// outer sweep) and the block pairs of the other rounds a cross sweep: every pair of columns is
// still rotated at least once per outer sweep, at about half the inner rounds.
__device__ __forceinline__ void inner_pair(int t, int i, bool full, int& a, int& b) {
  if (!full) { a = i; b = B + ((i + t) & (B - 1)); }
  else if (i == 0) { a = t; b = P - 1; }
  else { a = (t + i) % (P - 1); b = (t - i + (P - 1)) % (P - 1); }
}

// x (1 + cm) + y (ar + i ai) for complex x, y: the one-column form of every 2 x 2 rotation below,
// as three fused multiply-adds per component.
__device__ __forceinline__ float2 combo(float2 x, float2 y, float cm, float ar, float ai) {
  return make_float2(fmaf(-ai, y.y, fmaf(ar, y.x, fmaf(cm, x.x, x.x))),
                     fmaf(ai, y.x, fmaf(ar, y.y, fmaf(cm, x.y, x.y))));
}

// One cyclic two-sided Jacobi sweep on H (OFF_R1) accumulating Q (OFF_STAGE, fp32, starts as I):
// per round, 32 threads choose the rotations of the round's 32 disjoint pairs; then
// H <- J^* H J by 2 x 2 blocks (P <= P') and Q <- Q J, J = [[1 + cm1, es], [-conj(es), 1 + cm1]]
// per pair. A thread's blocks (P, P') are fixed for the sweep; their columns in round t follow from
// the schedule (inner_pair). Returns this thread's count of rotations.
__device__ int inner_sweep(unsigned char* sm, float tol2, bool full) {
  constexpr int NBLK = (528 + THREADS - 1) / THREADS;       // 2 x 2-block pairs (P, P') per thread
  float2* H = reinterpret_cast<float2*>(sm + OFF_R1);
  float2* Q = reinterpret_cast<float2*>(sm + OFF_STAGE);
  float4* prm = reinterpret_cast<float4*>(sm + OFF_PRM);
  const uint16_t* tri = reinterpret_cast<const uint16_t*>(sm + OFF_TRI);
  Misc* ms = misc(sm);
  for (int e = threadIdx.x; e < P * P; e += THREADS)
    Q[e] = make_float2((e / P) == (e % P) ? 1.f : 0.f, 0.f);
  int mp[NBLK], mq[NBLK];
#pragma unroll
  for (int k = 0; k < NBLK; ++k) {
    const int e = threadIdx.x + THREADS * k;
    const int v = e < 528 ? tri[e] : 0;
    mp[k] = e < 528 ? v >> 8 : -1;
    mq[k] = v & 0xff;
  }
  int nrot = 0;
  constexpr int QW = THREADS / 32;                          // rows of Q per pass
  const int qi = threadIdx.x & 31, qx = threadIdx.x >> 5;   // Q: pair qi, rows qx + QW k
  __syncthreads();
  const int rounds = full ? P - 1 : B;
  for (int t = 0; t < rounds; ++t) {
    if (threadIdx.x < 32) {
      int a, b;
      inner_pair(t, threadIdx.x, full, a, b);
      float al = H[a * HS + a].x, be = H[b * HS + b].x;
      const float2 g = H[a * HS + b];
      float gr = g.x, gi = g.y;
      const bool rot = pair_test(al, be, gr, gi, tol2);
      const float4 q = pair_params(al, be, gr, gi, rot);
      prm[threadIdx.x] = rot ? make_float4(q.x, q.y, q.z, 1.f) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (rot) { ++nrot; ms->rotated = 1; }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NBLK; ++k) {
      const int pp = mp[k], qq = mq[k];                     // pp <= qq
      if (pp < 0) continue;
      const float4 jp = prm[pp], jq = prm[qq];
      if (jp.w == 0.f && jq.w == 0.f) continue;
      int a, b, c, d;
      inner_pair(t, pp, full, a, b);
      inner_pair(t, qq, full, c, d);
      const float2 B00 = H[a * HS + c], B01 = H[a * HS + d], B10 = H[b * HS + c], B11 = H[b * HS + d];
      // T = B J_q: t0 = b0 (1 + cm) - b1 conj(es); t1 = b1 (1 + cm) + b0 es
      const float2 T00 = combo(B00, B01, jq.x, -jq.y, jq.z), T01 = combo(B01, B00, jq.x, jq.y, jq.z);
      const float2 T10 = combo(B10, B11, jq.x, -jq.y, jq.z), T11 = combo(B11, B10, jq.x, jq.y, jq.z);
      // B' = J_p^* T: row a' = (1 + cm) row_a - es row_b; row b' = (1 + cm) row_b + conj(es) row_a
      const float2 C00 = combo(T00, T10, jp.x, -jp.y, -jp.z), C01 = combo(T01, T11, jp.x, -jp.y, -jp.z);
      const float2 C10 = combo(T10, T00, jp.x, jp.y, -jp.z), C11 = combo(T11, T01, jp.x, jp.y, -jp.z);
      H[a * HS + c] = C00;
      H[a * HS + d] = C01;
      H[b * HS + c] = C10;
      H[b * HS + d] = C11;
      if (pp != qq) {
        H[c * HS + a] = make_float2(C00.x, -C00.y);
        H[d * HS + a] = make_float2(C01.x, -C01.y);
        H[c * HS + b] = make_float2(C10.x, -C10.y);
        H[d * HS + b] = make_float2(C11.x, -C11.y);
      }
    }
    {
      const float4 j = prm[qi];
      if (j.w != 0.f) {
        int a, b;
        inner_pair(t, qi, full, a, b);
        // every row's pair of entries first, then the rotated values (loads not held up by stores)
        float2 qa[P / QW], qb[P / QW];
#pragma unroll
        for (int k = 0; k < P / QW; ++k) {
          qa[k] = Q[(qx + QW * k) * P + a];
          qb[k] = Q[(qx + QW * k) * P + b];
        }
#pragma unroll
        for (int k = 0; k < P / QW; ++k) {
          const int x = qx + QW * k;
          Q[x * P + a] = combo(qa[k], qb[k], j.x, -j.y, j.z);   // qa (1 + cm) - qb conj(es)
          Q[x * P + b] = combo(qb[k], qa[k], j.x, j.y, j.z);    // qb (1 + cm) + qa es
        }
      }
    }
    __syncthreads();
  }
  return nrot;
}

// Q (OFF_STAGE, fp32 complex, Q[k][n] at k * 64 + n) -> the B operand of the update in its place
// (OFF_STAGE, 64 KB, over Q and the first half of H, both dead by then): the 128 x 64 (N x K) matrix
// [Re (Q - I)^T ; Im Q^T], rows n < 64 from Re(Q - I) and n >= 64 from Im Q, split into TF32 hi and lo
// (32 KB each), K-major core matrices (kc, ng) at byte ((kc * 16 + ng) * 8) * 16: LBO = 2048 B,
// SBO = 128 B. Layout: [hi | lo]. The update forms Y (Q - I) on the tensor cores and adds Y exactly
// on the CUDA cores: the 3xTF32 error (a few fp32 units of each product) then scales with the
// rotation, which is small once the sweeps near convergence, instead of with Y.
__device__ void q_to_operands(unsigned char* sm) {
  float2* Q = reinterpret_cast<float2*>(sm + OFF_STAGE);
  float* R = reinterpret_cast<float*>(sm + OFF_STAGE);
  constexpr int NQ = P * P / THREADS;
  float2 q[NQ];
#pragma unroll
  for (int j = 0; j < NQ; ++j) q[j] = Q[threadIdx.x + THREADS * j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    const int e = threadIdx.x + THREADS * j;
    const int k = e / P, n = e % P;
    const int off_re = ((k / 4 * 16 + n / 8) * 8 + n % 8) * 4 + k % 4;   // row n of B
    const int off_im = off_re + (P / 8) * 8 * 4;                          // row n + 64 of B
    float h, l;
    tc::split_tf32(k == n ? q[j].x - 1.f : q[j].x, h, l);
    R[off_re] = h;
    R[8192 + off_re] = l;
    tc::split_tf32(q[j].y, h, l);
    R[off_im] = h;
    R[8192 + off_im] = l;
  }
  tc::fence_proxy_async_smem();
  __syncthreads();
}

// ---------------------------------------------------------------------------------- update
// A matrix the update rewrites: column-major planes (re, im), leading dimension ld, `tiles` row
// tiles of RT rows.
struct Mat {
  float* re;
  float* im;
  int ld;
  int tiles;
};

// For every row tile of m0 and then of m1 (m1.tiles may be 0), the 64 columns cols[] of the tile
// become Y Q = Y + Y (Q - I). With B = [Re(Q - I) | Im Q] (N = 128), the tensor cores form
// D1 = Re Y B and D2 = Im Y B (TMEM columns [0, 128) and [128, 256)), and the CUDA cores add
//   Re Y' = Re Y + D1[:, c] - D2[:, 64 + c],   Im Y' = Im Y + D1[:, 64 + c] + D2[:, c].
// The work is a flat sequence of steps (tile, chunk of KU = 8 columns of Y): thread (row r, quad kc)
// loads Re and Im of row r of the chunk's columns 4 kc .. 4 kc + 3, keeps them for the tile's
// epilogue, and stages them as Re Y hi | lo | Im Y hi | lo (4 KB each, core matrix (kc, rg) at byte
// ((kc * 16 + rg) * 8) * 16: LBO = 2048 B, SBO = 128 B) in one of two buffers, PD chunks ahead of
// their loads. After the tile's last chunk each thread reads its 32 output columns' four
// accumulators out of TMEM (its row is its TMEM lane) and writes Y' with the Y it kept: no reload.
__device__ void update_pair(unsigned char* sm, Mat m0, Mat m1, const int* cols, Counters* ctr, uint32_t& ph) {
  static_assert(THREADS == 256 && KU == 8 && P / KU == 8, "each thread keeps a row's column quad per chunk");
  constexpr int PD = 2;                                 // chunks whose loads are in flight
  constexpr int CH = P / KU;                            // chunks per tile
  Misc* ms = misc(sm);
  float* const stage = reinterpret_cast<float*>(sm + OFF_UPD);
  const uint32_t s_base = tc::smem_u32(sm + OFF_UPD);
  const uint32_t q_base = tc::smem_u32(sm + OFF_STAGE);
  constexpr uint32_t LBO = 2048, SBO = 128;
  constexpr uint32_t PART = RT * KU * 4;                // bytes of one plane part (hi or lo, Re or Im)
  constexpr uint32_t ID = tc::idesc_tf32(128, 128);
  const int row = threadIdx.x & (RT - 1);
  const int kc = threadIdx.x >> 7;                      // this thread's column quad within a chunk
  const int tiles = m0.tiles + m1.tiles;
  const int soff = ((kc * 16 + (row >> 3)) * 8 + (row & 7)) * 4;
  auto load = [&](int T, int u, float* vr, float* vi) {
    const bool first = T < m0.tiles;
    const float* re = first ? m0.re : m1.re;
    const float* im = first ? m0.im : m1.im;
    const size_t ld = (size_t)(first ? m0.ld : m1.ld);
    const size_t r = (size_t)(first ? T : T - m0.tiles) * RT + row;
    const int c0 = u * KU + 4 * kc;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      vr[q] = __ldcg(re + (size_t)cols[c0 + q] * ld + r);
      vi[q] = __ldcg(im + (size_t)cols[c0 + q] * ld + r);
    }
  };
  auto stage_quad = [&](float* st, const float* v) {    // hi at st, lo one part further
    float4 h, l;
    tc::split_tf32(v[0], h.x, l.x);
    tc::split_tf32(v[1], h.y, l.y);
    tc::split_tf32(v[2], h.z, l.z);
    tc::split_tf32(v[3], h.w, l.w);
    *reinterpret_cast<float4*>(st + soff) = h;
    *reinterpret_cast<float4*>(st + PART / 4 + soff) = l;
  };
  float yr[CH][4], yi[CH][4];                           // this thread's Y of the current tile
  float nr[PD][4], ni[PD][4];                           // the next tile's first chunks, in flight
#pragma unroll
  for (int u = 0; u < PD; ++u) load(0, u, yr[u], yi[u]);
  int s = 0;
  for (int T = 0; T < tiles; ++T) {
#pragma unroll
    for (int u = 0; u < CH; ++u, ++s) {
      if (u + PD < CH) load(T, u + PD, yr[u + PD], yi[u + PD]);
      else if (T + 1 < tiles) load(T + 1, u + PD - CH, nr[u + PD - CH], ni[u + PD - CH]);
      const int b = s & 1;
      if (s >= 2) wait_buf(sm, ctr, b, ph);             // the MMAs of step s - 2 released buffer b
      float* st = stage + b * (4 * PART / 4);
      stage_quad(st, yr[u]);
      stage_quad(st + 2 * PART / 4, yi[u]);
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      if (threadIdx.x == 0 && !ms->failed) {
        tc::fence_after_sync();
        const uint32_t d1 = ms->tmem, d2 = ms->tmem + 128;
        const uint32_t a0 = s_base + (uint32_t)b * 4 * PART;
        const uint64_t yrh = tc::smem_desc_kmajor(a0, LBO, SBO);
        const uint64_t yrl = tc::smem_desc_kmajor(a0 + PART, LBO, SBO);
        const uint64_t yih = tc::smem_desc_kmajor(a0 + 2 * PART, LBO, SBO);
        const uint64_t yil = tc::smem_desc_kmajor(a0 + 3 * PART, LBO, SBO);
        const uint32_t qo = (uint32_t)(u * KU / 4) * LBO;
        const uint64_t bh = tc::smem_desc_kmajor(q_base + qo, LBO, SBO);
        const uint64_t bl = tc::smem_desc_kmajor(q_base + 32768 + qo, LBO, SBO);
        const uint32_t acc0 = u > 0 ? 1u : 0u;
        tc::mma_tf32(d1, yrh, bh, ID, acc0);             // D1 = Re Y B
        tc::mma_tf32(d1, yrh, bl, ID, 1u);
        tc::mma_tf32(d1, yrl, bh, ID, 1u);
        tc::mma_tf32(d2, yih, bh, ID, acc0);             // D2 = Im Y B
        tc::mma_tf32(d2, yih, bl, ID, 1u);
        tc::mma_tf32(d2, yil, bh, ID, 1u);
        tc::mma_commit(&ms->mbar[b]);
        if (u == CH - 1) tc::mma_commit(&ms->mbar[MB_TILE]);
      }
    }
    // epilogue of tile T: every MMA of the tile has completed
    wait_buf(sm, ctr, MB_TILE, ph);
    {
      const bool first = T < m0.tiles;
      float* Yr = first ? m0.re : m1.re;
      float* Yi = first ? m0.im : m1.im;
      const size_t ld = (size_t)(first ? m0.ld : m1.ld);
      const size_t r = (size_t)(first ? T : T - m0.tiles) * RT + row;
      const uint32_t ta = ms->tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16);
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const uint32_t c = (uint32_t)(u * KU + 4 * kc);
        float a[4], bq[4], cq[4], dq[4];
        tc::tmem_ld4(ta + c, a);               // D1[:, c]        Re Y Re(Q - I)
        tc::tmem_ld4(ta + 64 + c, bq);         // D1[:, 64 + c]   Re Y Im Q
        tc::tmem_ld4(ta + 128 + c, cq);        // D2[:, c]        Im Y Re(Q - I)
        tc::tmem_ld4(ta + 192 + c, dq);        // D2[:, 64 + c]   Im Y Im Q
        tc::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const size_t o = (size_t)cols[c + q] * ld + r;
          Yr[o] = yr[u][q] + (a[q] - dq[q]);
          Yi[o] = yi[u][q] + (bq[q] + cq[q]);
        }
      }
      tc::fence_before_sync();
      __syncthreads();                                  // the accumulators are free for the next tile
    }
#pragma unroll
    for (int u = 0; u < PD; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        yr[u][q] = nr[u][q];
        yi[u][q] = ni[u][q];
      }
  }
  // the operand buffers' last two commits (complete by now): one wait per commit keeps the parities
  for (int t = s >= 2 ? s - 2 : 0; t < s; ++t) wait_buf(sm, ctr, t & 1, ph);
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
    tc::mbar_init(&ms->mbar[0], 1);
    tc::mbar_init(&ms->mbar[1], 1);
    tc::mbar_init(&ms->mbar[MB_TILE], 1);
    tc::fence_mbar_init();
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

// ---------------------------------------------------------------------------------- warm start
// X = T W for a warm start (T, X: Mp x Np; W: Np x Np; complex, column-major planes, T and X with
// leading dimension ldx, W with ldw), on the CUDA cores in FP32. Only the first K columns of T and
// rows of W are nonzero (K a multiple of 32). 64 x 64 output tiles, K in chunks of 32 staged in
// shared memory (the block-pair region, free at the start of a symbol); thread (ty, tx) of 16 x 16
// forms the 4 x 4 complex block at rows 4 ty.., columns 4 tx...
__device__ void warm_gemm(unsigned char* sm, const float* Tr, const float* Ti, const float* Wr, const float* Wi,
                          float* Xr, float* Xi, int ldx, int ldw, int Mp, int Np, int K) {
  constexpr int TR = 64, TC = 64, TK = 32, SA = TR + 4, SB = TC + 4;
  static_assert(THREADS == 256 && 2 * TK * (SA + SB) * 4 <= REGION_BYTES, "tiles fit the region");
  float* sAr = reinterpret_cast<float*>(sm + OFF_STAGE);   // [TK][SA]: column k of the T tile
  float* sAi = sAr + TK * SA;
  float* sBr = sAi + TK * SA;                               // [TK][SB]: row k of the W tile
  float* sBi = sBr + TK * SB;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  for (int r0 = 0; r0 < Mp; r0 += TR) {
    for (int c0 = 0; c0 < Np; c0 += TC) {
      float accr[4][4], acci[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = 0.f;
      for (int k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
        for (int it = 0; it < TK * TR / THREADS; ++it) {   // T: 64 consecutive rows of column k
          const int e = threadIdx.x + THREADS * it, k = e / TR, r = e % TR;
          const size_t g = (size_t)(k0 + k) * ldx + r0 + r;
          sAr[k * SA + r] = __ldcg(Tr + g);
          sAi[k * SA + r] = __ldcg(Ti + g);
        }
#pragma unroll
        for (int it = 0; it < TK * TC / THREADS; ++it) {   // W: 32 consecutive rows of column c
          const int e = threadIdx.x + THREADS * it, c = e / TK, k = e % TK;
          const size_t g = (size_t)(c0 + c) * ldw + k0 + k;
          sBr[k * SB + c] = __ldcg(Wr + g);
          sBi[k * SB + c] = __ldcg(Wi + g);
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < TK; ++k) {
          const float4 ar = *reinterpret_cast<const float4*>(sAr + k * SA + 4 * ty);
          const float4 ai = *reinterpret_cast<const float4*>(sAi + k * SA + 4 * ty);
          const float4 br = *reinterpret_cast<const float4*>(sBr + k * SB + 4 * tx);
          const float4 bi = *reinterpret_cast<const float4*>(sBi + k * SB + 4 * tx);
          const float xr[4] = {ar.x, ar.y, ar.z, ar.w}, xi[4] = {ai.x, ai.y, ai.z, ai.w};
          const float yr[4] = {br.x, br.y, br.z, br.w}, yi[4] = {bi.x, bi.y, bi.z, bi.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              accr[i][j] = fmaf(xr[i], yr[j], fmaf(-xi[i], yi[j], accr[i][j]));
              acci[i][j] = fmaf(xr[i], yi[j], fmaf(xi[i], yr[j], acci[i][j]));
            }
        }
        __syncthreads();
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const size_t g = (size_t)(c0 + 4 * tx + j) * ldx + r0 + 4 * ty;
        *reinterpret_cast<float4*>(Xr + g) = make_float4(accr[0][j], accr[1][j], accr[2][j], accr[3][j]);
        *reinterpret_cast<float4*>(Xi + g) = make_float4(acci[0][j], acci[1][j], acci[2][j], acci[3][j]);
      }
    }
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

// One symbol per CTA (a persistent grid pulling symbols from an atomic work queue). Per symbol:
// assembly of X = A_k (or A_k^*) into the CTA's workspace slot and W = I, or with a warm start
// W = the previous symbol's V and X = A_k W (neighbouring frequencies have nearby singular
// vectors, so X starts nearly orthogonal and needs fewer sweeps); sweeps over the block
// pairs in circle-method order (nb - 1 rounds of nb / 2 pairs); then sigma, ranks and the
// normalised factors written to the layer's outputs. CTAs of 256 threads, two per SM.
template <bool VEC>
__global__ void __maxnreg__(bj::MAX_REGS) bj_kernel(const __grid_constant__ BJLaunch A) {
  using namespace bj;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ int scols[P];
  __shared__ float sinv[2][P];          // 1/|x_c| (0 for a negligible column), 1/|w_c| of 64 columns
  __shared__ int srank[P];
  Counters* ctr = A.counters;
  const int Mp = A.Mp, Np = A.Np, ldx = A.ldx, ldw = A.ldw;
  const int nb = Np / B;
  float* Xr = A.ws + (size_t)blockIdx.x * A.slot_floats;
  float* Xi = Xr + (size_t)Np * ldx;
  float* Wr = Xi + (size_t)Np * ldx;
  float* Wi = Wr + (size_t)Np * ldw;
  float* sg = VEC ? Wi + (size_t)Np * ldw : Wr;   // sigma of every column of the symbol
  float2* phs = reinterpret_cast<float2*>(sm + OFF_PHS);
  Misc* ms = misc(sm);
  cta_setup(sm);
  uint32_t ph = 0;   // mbarrier phase parities (see wait_buf)
  unsigned int* queue = &ctr->queue[A.queue_slot];

  // phase clocks of thread 0: Gram, inner sweep, update, assembly, output, whole symbols
  // kept in shared memory by thread 0 (no registers held across the phases)
  __shared__ unsigned long long cyc[6];
  __shared__ long long c_sym, c_ph;
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) cyc[k] = 0;
  for (;;) {
    if (threadIdx.x == 0) ms->item = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int item = ms->item;
    if (item >= A.total_items) break;
    // item t: run t % runs, position t / runs in it, symbol g = run * run_len + position of the launch
    int g = item, pos = 0;
    if (A.runs > 0) {
      pos = item / A.runs;
      g = (item - pos * A.runs) * A.run_len + pos;
      if (g >= A.total_symbols) {                       // past the launch's last symbol
        __syncthreads();                                // every thread has read ms->item
        continue;
      }
    }
    int lk = 0;                                         // the symbol's layer
    while (lk + 1 < A.nlayers && g >= A.L[lk + 1].item_begin) ++lk;
    const LayerArgs& La = A.L[lk];
    const int h = g - La.item_begin;                    // half-grid symbol of that layer
    if (!LFA_DOK(La.dbg, h >= 0 && h < La.F_h, 5)) {   // blocked route: item -> layer, symbol
      __syncthreads();                                 // every thread has read ms->item
      continue;
    }
    const int M = La.M, N = La.N;
    if (threadIdx.x == 0) {
      c_sym = clock64();
      // a warm start when the run's previous symbol is done (its factors are in the outputs)
      // (the previous symbol of the run in the same layer)
      ms->warm = (VEC && pos > 0 && h > 0 && tc::ld_acquire_gpu(A.done + g - 1) != 0) ? 1 : 0;
    }
    const int f = La.half[h];
    const int jj = f / La.m, ll = f - jj * La.m;
    const int kk = La.kh * La.kw;
    for (int t = threadIdx.x; t < kk; t += THREADS) phs[t] = tap_phase(La, jj, ll, t / La.kw, t % La.kw);
    __syncthreads();
    const bool warm = VEC && ms->warm;
    // ---- X = the symbol (assembled from the taps), W = I; padding rows and columns are zero.
    // Warm start: the symbol goes to the T planes, W = V of the run's previous symbol, X = T W (the
    // sweeps keep X = A W for any starting W; a nearly orthogonal T W needs fewer of them)
    float* Tr = warm ? sg + Np : Xr;
    float* Ti = warm ? Tr + (size_t)Np * ldx : Xi;
    for (int c = 0; c < Np; ++c) {
      for (int row = threadIdx.x; row < Mp; row += THREADS) {
        const float2 v = x_entry<true>(La, h, row, c, phs);
        Tr[(size_t)c * ldx + row] = v.x;
        Ti[(size_t)c * ldx + row] = v.y;
      }
      if constexpr (VEC) {
        if (!warm) {
          for (int row = threadIdx.x; row < Np; row += THREADS) {
            Wr[(size_t)c * ldw + row] = (row == c && c < N) ? 1.f : 0.f;
            Wi[(size_t)c * ldw + row] = 0.f;
          }
        }
      }
    }
    if constexpr (VEC) {
      if (warm) {
        // W(row, c) = Wo(row, c) of the previous symbol (row-major N x N, read along rows)
        const float2* Wp = (La.wide ? La.U : La.V) + (size_t)(h - 1) * N * N;
        for (int e = threadIdx.x; e < Np * Np; e += THREADS) {
          const int row = e / Np, c = e - row * Np;
          const float2 v = (row < N && c < N) ? __ldcg(Wp + (size_t)row * N + c) : make_float2(0.f, 0.f);
          Wr[(size_t)c * ldw + row] = v.x;
          Wi[(size_t)c * ldw + row] = v.y;
        }
        __syncthreads();
        warm_gemm(sm, Tr, Ti, Wr, Wi, Xr, Xi, ldx, ldw, Mp, Np, (N + 31) / 32 * 32);
        if (threadIdx.x == 0) atomicAdd(&ctr->warm_starts, 1ull);
      }
    }
    __threadfence_block();
    __syncthreads();
    if (threadIdx.x == 0) {
      c_ph = clock64();
      cyc[3] += (unsigned long long)(c_ph - c_sym);
    }
    // ---- sweeps
    int sweeps = 0, nrot = 0, ngram = 0, nupd = 0;
    bool converged = false;
    for (;;) {
      int rotated_sweep = 0;
      for (int t = 0; t < nb - 1; ++t) {
        for (int pos = 0; pos < nb / 2; ++pos) {
          int I, J;
          outer_pair(t, pos, nb, I, J);
          if (threadIdx.x < P) scols[threadIdx.x] = threadIdx.x < B ? I * B + threadIdx.x : J * B + threadIdx.x - B;
          if (threadIdx.x == 0) ms->rotated = 0;
          __syncthreads();
          gram_pair(sm, Xr, Xi, ldx, Mp, scols, ctr, ph);
          const bool full = (t == 0);         // the first round of the sweep: intra-block pairs too
          gram_to_h(sm, La.tol2, full);
          ++ngram;
          if (threadIdx.x == 0) {
            const long long c1 = clock64();
            cyc[0] += (unsigned long long)(c1 - c_ph);
            c_ph = c1;
          }
          if (ms->any) {                      // else no pair of the block pair rotates: skip the rest
            nrot += inner_sweep(sm, La.tol2, full);
            if (threadIdx.x == 0) {
              const long long c1 = clock64();
              cyc[1] += (unsigned long long)(c1 - c_ph);
              c_ph = c1;
            }
            if (ms->rotated) {
              rotated_sweep = 1;
              ++nupd;
              q_to_operands(sm);
              update_pair(sm, Mat{Xr, Xi, ldx, Mp / RT}, Mat{Wr, Wi, ldw, VEC ? Np / RT : 0}, scols, ctr, ph);
            }
          }
          __syncthreads();
          if (threadIdx.x == 0) {
            const long long c1 = clock64();
            cyc[2] += (unsigned long long)(c1 - c_ph);
            c_ph = c1;
          }
        }
      }
      ++sweeps;
      if (!rotated_sweep) { converged = true; break; }
      if (sweeps >= A.max_sweeps) break;
    }
    if (threadIdx.x == 0) {
      atomicAdd(&ctr->sweeps, (unsigned long long)sweeps);
      atomicAdd(&ctr->tc_grams, (unsigned long long)ngram);
      atomicAdd(&ctr->tc_updates, (unsigned long long)nupd);
      if (!converged) atomicAdd(&ctr->unconverged, 1ull);
    }
    if (threadIdx.x < 32 && nrot) atomicAdd(&ctr->rotations, (unsigned long long)nrot);
    // ---- sigma_c = |x_c| / |w_c| (x_c = A w_c to rounding), 64 columns at a time
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < Np; c0 += P) {
      for (int cl_ = w; cl_ < P; cl_ += THREADS / 32) {
        const int c = c0 + cl_;
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
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          xn += __shfl_xor_sync(0xffffffffu, xn, o);
          wn += __shfl_xor_sync(0xffffffffu, wn, o);
        }
        if constexpr (!VEC) wn = 1.f;   // values only: W is not tracked, |w_c| = 1
        const float ixn = xn > 0x1p-100f ? rsqrt_nr(xn) : 0.f;   // the sweeps' zero-column bound
        const float iwn = wn > 0.f ? rsqrt_nr(wn) : 0.f;
        if (lane == 0) sg[c] = c < N ? xn * ixn * iwn : -1.f;
      }
    }
    __threadfence_block();
    __syncthreads();
    // ---- ranks (descending sigma, ties by column index), sigma, and the normalised factors
    float2* Xo = VEC ? (La.wide ? La.V : La.U) + (size_t)h * M * N : nullptr;
    float2* Wo = VEC ? (La.wide ? La.U : La.V) + (size_t)h * N * N : nullptr;
    for (int c0 = 0; c0 < N; c0 += P) {
      if (threadIdx.x < P) {
        const int c = c0 + threadIdx.x;
        int rank = -1;
        if (c < N) {
          const float sc = __ldcg(sg + c);
          bool finite = true;
          float smax = 0.f;
          rank = 0;
          for (int q2 = 0; q2 < N; ++q2) {
            const float v = __ldcg(sg + q2);
            finite = finite && isfinite(v);
            smax = fmaxf(smax, v);
            rank += (v > sc) || (v == sc && q2 < c);
          }
          float* srow = La.sigma + (size_t)(A.half_output ? h : f) * La.r;
          if (LFA_DOK(La.dbg, rank >= 0 && rank < N, 6)) srow[rank] = sc;   // blocked route: rank
          if (!A.half_output) {
            const int fc = ((La.n - jj) % La.n) * La.m + (La.m - ll) % La.m;
            if (fc != f) La.sigma[(size_t)fc * La.r + rank] = sc;
          }
          if (c == 0 && !finite) atomicAdd(&ctr->nonfinite, 1ull);
          // a column far below sigma_max carries no direction: written as zero, completed afterwards
          sinv[0][threadIdx.x] = (sc > 1e-12f * smax) ? 1.f : 0.f;
        }
        srank[threadIdx.x] = rank;
      }
      __syncthreads();
      if constexpr (VEC) {
        for (int cl_ = w; cl_ < P; cl_ += THREADS / 32) {
          const int c = c0 + cl_, rk = srank[cl_];
          if (rk < 0) continue;
          // column norms once more (a warp per column), then the normalised columns
          float xn = 0.f, wn = 0.f;
          for (int row = lane; row < Mp; row += 32) {
            const float a = __ldcg(Xr + (size_t)c * ldx + row), b = __ldcg(Xi + (size_t)c * ldx + row);
            xn = fmaf(a, a, fmaf(b, b, xn));
          }
          for (int row = lane; row < Np; row += 32) {
            const float a = __ldcg(Wr + (size_t)c * ldw + row), b = __ldcg(Wi + (size_t)c * ldw + row);
            wn = fmaf(a, a, fmaf(b, b, wn));
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            xn += __shfl_xor_sync(0xffffffffu, xn, o);
            wn += __shfl_xor_sync(0xffffffffu, wn, o);
          }
          const float ix = (xn > 0x1p-100f ? rsqrt_nr(xn) : 0.f) * sinv[0][cl_];
          const float iw = wn > 0.f ? rsqrt_nr(wn) : 0.f;
          for (int row = lane; row < M; row += 32)
            Xo[(size_t)row * N + rk] = make_float2(__ldcg(Xr + (size_t)c * ldx + row) * ix,
                                                   __ldcg(Xi + (size_t)c * ldx + row) * ix);
          for (int row = lane; row < N; row += 32)
            Wo[(size_t)row * N + rk] = make_float2(__ldcg(Wr + (size_t)c * ldw + row) * iw,
                                                   __ldcg(Wi + (size_t)c * ldw + row) * iw);
        }
      }
      __syncthreads();
    }
    if (VEC && A.runs > 0) __threadfence();   // this thread's outputs, before the done flag
    __syncthreads();   // the slot is reused by the CTA's next symbol
    if (threadIdx.x == 0) {
      // every thread's outputs precede the barrier; the release publishes them with the flag
      if (VEC && A.runs > 0) tc::st_release_gpu(A.done + g, 1);
      const long long c_end = clock64();
      cyc[4] += (unsigned long long)(c_end - c_ph);
      cyc[5] += (unsigned long long)(c_end - c_sym);
    }
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) atomicAdd(&ctr->bj_cycles[k], cyc[k]);
  cta_teardown(sm);
}

int g_bj_ctas_per_sm = 0;
int g_bj_max_ctas = 0;
int g_bj_runs = 0;

template <bool VEC>
static cudaError_t bj_prepare_t(int sms, int* max_ctas) {
  cudaError_t e = cudaFuncSetAttribute(bj_kernel<VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bj::SMEM);
  if (e == cudaSuccess)   // all of the SM's unified memory as shared memory
    e = cudaFuncSetAttribute(bj_kernel<VEC>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess || !max_ctas) return e;
  int b = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, bj_kernel<VEC>, bj::THREADS, bj::SMEM);
  if (e != cudaSuccess) return e;
  // two CTAs of 256 threads per SM (each holds TMEM_COLS of the SM's 512 tensor-memory columns)
  const int per_sm = g_bj_ctas_per_sm > 0 ? std::min(g_bj_ctas_per_sm, bj::CTAS_PER_SM) : bj::CTAS_PER_SM;
  *max_ctas = (b >= 1 ? per_sm : 0) * sms;
  return cudaSuccess;
}

// The route serves 128 to 512 columns (fewer leave most of the 128-column padding idle) and up
// to 512 rows.
bool bj_supported(int M, int N) { return N >= 128 && M <= 512 && N <= 512; }

// The built-in choice takes the blocked route for tall or square symbols of 129-512 columns when a
// layer has enough symbols to fill the GPU. One symbol per CTA takes ~20 ms at 256 columns, ~55 ms
// at 384 and ~125 ms at 512 (alone on an SM, values), while the element-wise cluster kernels spread
// a symbol over up to 16 SMs at ~0.24, ~1.9 and ~1.9 ms of throughput per symbol (GB300): the
// blocked route is the faster one from about 84, 30 and 68 symbols.
int bj_min_symbols(int N) { return N <= 256 ? 84 : N <= 384 ? 30 : 68; }
void bj_dims(int M, int N, int* Mp, int* Np) {
  *Mp = (M + bj::RT - 1) / bj::RT * bj::RT;
  *Np = (N + 127) / 128 * 128;
}

template <bool VEC>
static cudaError_t bj_occupancy_t(int* blocks, int* regs, int* smem_static, int* smem_dyn) {
  cudaError_t e = bj_prepare_t<VEC>(0, nullptr);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, bj_kernel<VEC>);
  if (e != cudaSuccess) return e;
  *regs = fa.numRegs;
  *smem_static = (int)fa.sharedSizeBytes;
  *smem_dyn = bj::SMEM;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, bj_kernel<VEC>, bj::THREADS, bj::SMEM);
  if (e != cudaSuccess) return e;
  // the same with 32 KB of dynamic shared memory: tells a shared-memory limit from a register limit
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks + 1, bj_kernel<VEC>, bj::THREADS, 32768);
}

cudaError_t bj_occupancy(bool vec, int* blocks, int* regs, int* smem_static, int* smem_dyn) {
  return vec ? bj_occupancy_t<true>(blocks, regs, smem_static, smem_dyn)
             : bj_occupancy_t<false>(blocks, regs, smem_static, smem_dyn);
}

cudaError_t bj_max_ctas(bool vec, int sms, int* ctas) {
  return vec ? bj_prepare_t<true>(sms, ctas) : bj_prepare_t<false>(sms, ctas);
}

size_t bj_slot_floats(int M, int N, bool vec) {
  int Mp, Np;
  bj_dims(M, N, &Mp, &Np);
  // X planes, W planes (vectors), sigma per column, and with vectors a warm start's T planes
  return (size_t)2 * Np * Mp + (vec ? (size_t)2 * Np * Np : 0) + (size_t)Np + (vec ? (size_t)2 * Np * Mp : 0);
}

cudaError_t launch_bj(const BJLaunch& A, int ctas, bool vec, cudaStream_t s) {
  cudaError_t e = vec ? bj_prepare_t<true>(0, nullptr) : bj_prepare_t<false>(0, nullptr);
  if (e != cudaSuccess) return e;
  if (vec) bj_kernel<true><<<ctas, bj::THREADS, bj::SMEM, s>>>(A);
  else bj_kernel<false><<<ctas, bj::THREADS, bj::SMEM, s>>>(A);
  return cudaGetLastError();
}

// ================================================================================== debug kernels
// One CTA: the Gram of one block pair (the tensor-core contraction of the route), written out.
__global__ void __launch_bounds__(bj::THREADS, 1)
bj_gram_test_kernel(const float* Xr, const float* Xi, int ld, int Mp, const int* cols, float* D, Counters* ctr) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ int scol[bj::P];
  if (threadIdx.x < bj::P) scol[threadIdx.x] = cols[threadIdx.x];
  bj::cta_setup(sm);
  uint32_t ph = 0;
  bj::gram_pair(sm, Xr, Xi, ld, Mp, scol, ctr, ph);
  bj::gram_to_h(sm, 0.f, true);
  const float2* H = reinterpret_cast<const float2*>(sm + bj::OFF_R1);
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
  float2* Q = reinterpret_cast<float2*>(sm + bj::OFF_STAGE);
  for (int e = threadIdx.x; e < bj::P * bj::P; e += bj::THREADS) Q[e] = Qin[e];
  __syncthreads();
  bj::q_to_operands(sm);
  // the update rewrites its planes in place: copy the columns to the outputs first
  for (int e = threadIdx.x; e < bj::P * rows; e += bj::THREADS) {
    const size_t k = (size_t)scol[e / rows] * ld + e % rows;
    Or[k] = Pr[k];
    Oi[k] = Pi[k];
  }
  __threadfence_block();
  __syncthreads();
  uint32_t ph = 0;
  bj::update_pair(sm, bj::Mat{Or, Oi, ld, rows / bj::RT}, bj::Mat{Or, Oi, ld, 0}, scol, ctr, ph);
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
// 64, ld a multiple of 4); H written to D as complex64 [64][64]. Returns 0, or the CUDA error.
int32_t lfa_debug_tc_gram(const float* Xr, const float* Xi, int32_t ld, int32_t Mp, const int32_t* cols, float* D,
                          void* stream) {
  if (!Xr || !Xi || !cols || !D || ld < Mp || (ld & 3) || Mp < lfa::bj::KC || (Mp % lfa::bj::KC)) return -1;
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
