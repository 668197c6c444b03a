// Batched one-sided (Hestenes) Jacobi SVD of the LFA symbols, fused with symbol
// assembly (arXiv 2506.05617, Sec. III: symbol A_k = sum_y M_y exp(2 pi i <k,y>)
// and its SVD A_k = U_k S_k V_k^*, Algorithm 1 lines 4-5).
//
// Design (sm_103a):
//  * The N columns of X (X = A_k or A_k^*, M x N, N = r, padded to NC = 2 NP) are
//    paired; each pair is owned by a team of L lanes, each lane holding MR rows of
//    both columns of X (and WR rows of the accumulated rotations W) in registers.
//    Rows are interleaved: lane l holds rows l, l + L, l + 2L, ... A thread may serve
//    PPT = 2 teams, whose rounds are independent dependency chains it interleaves.
//  * One round: every team forms alpha = |x_p|^2, beta = |x_q|^2, gamma = x_p^* x_q
//    by an xor butterfly over its L lanes (bitwise identical on every lane, so the
//    team takes one decision) and, when |gamma| > tol sqrt(alpha beta), applies the
//    complex rotation that makes x_p, x_q orthogonal, to X and W.
//  * Rounds follow the circle-method round robin: at round t the pair at position i
//    is (c(t+i), c(t-i)) for i >= 1 and (c(t), NC-1) for i = 0, c(x) = x mod NC-1.
//    Between rounds the team at position i keeps one column and sends the other to
//    the neighbouring position (0 -> 1, odd i -> i-1, even i -> i+1); teams move by
//    the fixed involution pi = (1 2)(3 4)...(NP-3 NP-2), so team k sits at position k
//    on even rounds and pi(k) on odd ones. Each team receives exactly one column per
//    round into its own slot of a shared-memory mailbox (double-buffered by round
//    parity, so one barrier per round suffices). No schedule table is needed.
//  * With CS > 1 the teams of one symbol are spread over a thread-block cluster of CS
//    CTAs; columns move through distributed shared memory and the per-round barrier
//    is the cluster barrier. This keeps symbols up to 512 columns register-resident.
//  * Sweeps (NC-1 rounds) repeat until no pair of a sweep rotates (or max_sweeps).
//    sigma_p = |x_p| / |w_p| (recomputed), U (V for wide symbols) columns x_p/|x_p|,
//    the other factor w_p/|w_p|.
//  * Symbol assembly is fused: each lane assembles its own entries of X from the
//    weights (L1/L2) and the k_h x k_w phase grid of the frequency (shared memory).
//  * Work items (symbol tiles) come from an atomic queue: one persistent launch per
//    variant serves every layer of that variant.
#pragma once

#include <cooperative_groups.h>

#include "lfa_internal.cuh"

namespace lfa {

namespace cg = cooperative_groups;

template <int NP_, int L_, int MR_, int WR_, bool VEC_, int CS_, int MINB_ = 1, int PPT_ = 1>
struct JCfg {
  static constexpr int NP = NP_, L = L_, MR = MR_, WR = WR_, CS = CS_, PPT = PPT_;
  static constexpr bool VEC = VEC_;
  static_assert(NP % 2 == 0 && NP % CS == 0, "pairs must be even and split evenly over the cluster");
  static constexpr int TPC = NP / CS;             // teams per CTA
  static_assert(PPT == 1 || PPT == 2, "a thread holds rows of one or two teams");
  static_assert(TPC % PPT == 0, "teams split evenly over the threads");
  static constexpr int TC = TPC / PPT * L;        // threads per CTA per symbol
  static constexpr int UT = TC <= 32 ? 32 : TC;   // threads per unit (a warp, or the CTA)
  static constexpr int SPU = TC <= 32 ? 32 / TC : 1;
  static constexpr int BLOCK = TC <= 32 ? 128 : TC;
  static constexpr int UPB = BLOCK / UT;          // units per CTA
  static constexpr int NC = 2 * NP;               // column slots
  static constexpr int XR = MR * L;               // X row capacity
  static_assert(MR % 2 == 0, "X rows are held as pairs");
  static constexpr int MH = MR / 2;               // X row pairs per lane
  static constexpr int WH = (WR + 1) / 2;         // W row pairs per lane (last one half padding if WR odd)
  static constexpr int WRC = VEC ? 2 * WH * L : 0;  // W row capacity in the mailbox
  // slot stride = 2 L mod 16 (float2): a column moves as 16-byte (re, im) pairs, a shared-memory
  // phase serves 8 lanes, so the L lanes of neighbouring teams must be L * 16 bytes apart mod 128
  static constexpr int RS = XR + WRC + (((2 * L - (XR + WRC)) % 16) + 16) % 16;
  static_assert(RS % 2 == 0, "mailbox slots start on 16-byte boundaries");
  static constexpr int MBOX = 2 * TPC * RS;       // [parity][team][RS] float2
  static constexpr size_t SYM_BYTES = (size_t)(MBOX + kMaxTaps) * 8 + NC * 4 + 2 * TPC * 4 + 64;
  // unit tail: ubox[4] (item, sweep votes, zero-column count) + one float per warp of the unit
  // for unit_sum's reduction
  static constexpr size_t TAIL_BYTES = (16 + 4 * (UT / 32) + 15) / 16 * 16 < 64 ? 64 : (16 + 4 * (UT / 32) + 15) / 16 * 16;
  static constexpr size_t UNIT_BYTES = SPU * SYM_BYTES + TAIL_BYTES;
  static_assert(SYM_BYTES % 16 == 0 && UNIT_BYTES % 16 == 0, "every symbol's mailbox is 16-byte aligned");
  static_assert(!VEC || CS > 1 || XR <= kMaxTaps, "the in-kernel completion's row buffer fits the phase grid");
  static constexpr size_t SMEM = UPB * UNIT_BYTES;
  static constexpr int MINB = MINB_;   // resident CTAs per SM the register allocation aims for
  static_assert((size_t)NC * (XR + WRC) <= (size_t)MBOX || CS > 1, "staging must fit the mailbox");
};

template <int T>
__device__ __forceinline__ unsigned sym_mask(int sym) {
  if constexpr (T >= 32) return 0xffffffffu;
  else return ((1u << T) - 1u) << ((sym * T) & 31);
}

template <int L>
__device__ __forceinline__ float team_sum(float v) {
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Barrier over the threads that share a symbol's data (warp, CTA or cluster).
template <class C>
__device__ __forceinline__ void sym_sync() {
  if constexpr (C::CS > 1) cg::this_cluster().sync();
  else if constexpr (C::UT == 32) __syncwarp();
  else __syncthreads();
}

// Barrier over the threads of this CTA's unit.
template <class C>
__device__ __forceinline__ void unit_sync() {
  if constexpr (C::UT == 32) __syncwarp();
  else __syncthreads();
}

// Sum over the UT threads of a unit (all threads must call it).
template <class C>
__device__ __forceinline__ float unit_sum(float v, float* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if constexpr (C::UT == 32) {
    return v;
  } else {
    const int wid = (threadIdx.x % C::UT) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[wid] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < C::UT / 32; ++i) s += red[i];
    return s;
  }
}

// The fixed team movement between rounds: (1 2)(3 4)...(NP-3 NP-2); 0 and NP-1 stay.
template <int NP>
__device__ __forceinline__ int pi_pos(int p) {
  if (p == 0 || p == NP - 1) return p;
  return (p & 1) ? p + 1 : p - 1;
}

// Entry X[row][col] of the symbol (phases in `phs`), or 0 outside M x N.
template <bool FUSED>
__device__ __forceinline__ float2 x_entry(const LayerArgs& La, int h, int row, int col,
                                          const float2* phs) {
  if (row >= La.M || col >= La.N) return make_float2(0.f, 0.f);
  const int o = La.wide ? col : row;
  const int i = La.wide ? row : col;
  float2 v;
  if constexpr (FUSED) v = symbol_entry(La, o, i, phs);
  else v = La.symbols[((size_t)h * La.c_out + o) * La.c_in + i];
  return make_float2(v.x, La.wide ? -v.y : v.y);
}

// A column of X (and of W) held by one lane as real/imaginary planes over row pairs: pair k
// holds rows lane + L k (.x) and lane + L (k + MH) (.y) of X; for W the pair partner row is
// lane + L (k + WH). Every complex operation on a column is then an elementwise operation on
// pairs, issued as paired fp32 instructions (two fused multiply-adds per instruction).
template <class C>
struct Planes {
  float2 xr[C::MH], xi[C::MH];
  float2 wr[C::VEC ? C::WH : 1], wi[C::VEC ? C::WH : 1];
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// 1/sqrt(x) for normal x > 0: the hardware estimate refined by one Newton-Raphson step for
// the reciprocal square root, y <- y (3 - x y^2) / 2, which brings it to about one ulp. The
// rotation's unitarity rests on e = gamma/|gamma| and s having unit modulus to this accuracy.
__device__ __forceinline__ float rsqrt_nr(float x) {
  const float y = rsqrtf(x);
  const float h = 0.5f * x * y;
  return fmaf(y, fmaf(-h, y, 0.5f), y);   // y + y (1/2 - x y^2 / 2)
}

// One Jacobi round on a team's pair (a, b) comes in three phases, so that a thread holding two
// pairs can interleave their dependency chains: pair_dots (alpha = |a|^2, beta = |b|^2,
// gamma = a^* b, summed over the team's L lanes, bitwise identical on every lane), pair_test
// (scaling and the rotation test), pair_params (the rotation) and rotate_pair (X and W).
template <class C>
__device__ __forceinline__ void pair_dots(const Planes<C>& a, const Planes<C>& b, float& al, float& be,
                                          float& gr, float& gi) {
  constexpr int MH = C::MH, L = C::L;
  // real and imaginary planes accumulate separately: eight independent chains
  float2 alr = f2(0.f), ali = f2(0.f), ber = f2(0.f), bei = f2(0.f);
  float2 grr = f2(0.f), gri = f2(0.f), gp2 = f2(0.f), gm2 = f2(0.f);
#pragma unroll
  for (int k = 0; k < MH; ++k) {
    alr = __ffma2_rn(a.xr[k], a.xr[k], alr);
    ali = __ffma2_rn(a.xi[k], a.xi[k], ali);
    ber = __ffma2_rn(b.xr[k], b.xr[k], ber);
    bei = __ffma2_rn(b.xi[k], b.xi[k], bei);
    grr = __ffma2_rn(a.xr[k], b.xr[k], grr);   // Re(conj(a) b) = ar br + ai bi
    gri = __ffma2_rn(a.xi[k], b.xi[k], gri);
    gp2 = __ffma2_rn(a.xr[k], b.xi[k], gp2);   // Im(conj(a) b) = ar bi - ai br
    gm2 = __ffma2_rn(a.xi[k], b.xr[k], gm2);
  }
  const float2 al2 = __fadd2_rn(alr, ali), be2 = __fadd2_rn(ber, bei), gr2 = __fadd2_rn(grr, gri);
  al = al2.x + al2.y;
  be = be2.x + be2.y;
  gr = gr2.x + gr2.y;
  gi = (gp2.x + gp2.y) - (gm2.x + gm2.y);
  al = team_sum<L>(al);
  be = team_sum<L>(be);
  gr = team_sum<L>(gr);
  gi = team_sum<L>(gi);
}

// Scales the pair's quantities (in place) and decides whether it rotates.
__device__ __forceinline__ bool pair_test(float& al, float& be, float& gr, float& gi, float tol2) {
  // The rotation depends only on ratios, so scale the pair by a power of two that brings the
  // larger squared norm into [1, 4): |gamma|^2 then stays a normal float down to column-norm
  // ratios of ~1e-19. Without it, columns of a rank-deficient symbol shrink by ~eps every sweep
  // (they are re-projected against the others), |gamma|^2 goes denormal, e = gamma/|gamma| loses
  // its unit modulus and the rotations stop being unitary.
  // Both squared norms below 2^-100: the columns are zero. Above it their entries' products
  // are normal floats, so |gamma| is exact enough for the threshold test (below it, denormal
  // products leave gamma ~1e-5 relative noise and such a pair would rotate every sweep).
  const float mx = fmaxf(al, be);
  const int ex = (__float_as_int(mx) >> 23) & 0xff;  // biased exponent of mx
  const float sc = __int_as_float(max(254 - ex, 1) << 23);
  al *= sc;
  be *= sc;
  gr *= sc;
  gi *= sc;
  const float g2 = fmaf(gr, gr, gi * gi);
  // a denormal |gamma|^2 that passes the test has be < 2e-25 al: the angle is below 1e-19
  return mx >= 0x1p-100f && g2 > tol2 * (al * be) && g2 >= 1.17549435e-38f;
}

// Rotation parameters (c-1, Re(e s), Im(e s)) from the scaled quantities. With rot = false the
// inputs are replaced by harmless ones, so the call may run unconditionally (its result unused).
__device__ __forceinline__ float4 pair_params(float al, float be, float gr, float gi, bool rot) {
  if (!rot) { al = 0.f; be = 0.f; gr = 1.f; gi = 0.f; }
  const float g2 = fmaf(gr, gr, gi * gi);
  // J = [[c, s e], [-s conj(e), c]], e = gamma/|gamma|, t = tan solves t^2 + 2 zeta t - 1 = 0
  // with zeta = (beta - alpha)/(2|gamma|), |t| <= 1. The angle may be approximate; unitarity
  // rests on e, s and c-1, which are formed with correctly rounded reciprocals / reciprocal
  // square roots. Applied as x + (c-1) x + ...: c - 1 = -t^2/(r(1+r)), r = sqrt(1+t^2) (for
  // small t fp32 rounds c to 1, and c = 1, s = t would grow norms by t^2/2).
  const float ig = rsqrt_nr(g2);                     // 1/|gamma|
  const float zeta = (be - al) * (0.5f * ig);
  const float az = fabsf(zeta);
  const float q = fmaf(az, az, 1.f);
  const float hz = az < 1e18f ? q * rsqrtf(q) : az;  // ~ sqrt(1 + zeta^2)
  const float tt = copysignf(__fdividef(1.f, az + hz), zeta);
  const float r2 = fmaf(tt, tt, 1.f);
  const float ir = rsqrt_nr(r2);
  const float s = tt * ir;
  const float r = r2 * ir;
  const float cm1 = __fdividef(-(tt * s), 1.f + r);  // tiny for small t: its relative error is harmless
  return make_float4(cm1, s * (gr * ig), s * (gi * ig), 0.f);
}

// a' = a + (c-1) a - conj(e s) b ; b' = b + (c-1) b + (e s) a,  e s = sr + i si:
//   a'r = ar + cm1 ar - sr br - si bi     a'i = ai + cm1 ai - sr bi + si br
//   b'r = br + cm1 br + sr ar - si ai     b'i = bi + cm1 bi + sr ai + si ar
// on the X planes and, with vectors, on the W planes.
template <class C>
__device__ __forceinline__ void rotate_pair(Planes<C>& a, Planes<C>& b, float4 prm) {
  constexpr int MH = C::MH, WH = C::WH;
  const float2 c2 = f2(prm.x), s2 = f2(prm.y), ns2 = f2(-prm.y), t2 = f2(prm.z), nt2 = f2(-prm.z);
#pragma unroll
  for (int k = 0; k < MH; ++k) {
    const float2 Ar = a.xr[k], Ai = a.xi[k], Br = b.xr[k], Bi = b.xi[k];
    a.xr[k] = __ffma2_rn(nt2, Bi, __ffma2_rn(ns2, Br, __ffma2_rn(c2, Ar, Ar)));
    a.xi[k] = __ffma2_rn(t2, Br, __ffma2_rn(ns2, Bi, __ffma2_rn(c2, Ai, Ai)));
    b.xr[k] = __ffma2_rn(nt2, Ai, __ffma2_rn(s2, Ar, __ffma2_rn(c2, Br, Br)));
    b.xi[k] = __ffma2_rn(t2, Ar, __ffma2_rn(s2, Ai, __ffma2_rn(c2, Bi, Bi)));
  }
  if constexpr (C::VEC) {
#pragma unroll
    for (int k = 0; k < WH; ++k) {
      const float2 Ar = a.wr[k], Ai = a.wi[k], Br = b.wr[k], Bi = b.wi[k];
      a.wr[k] = __ffma2_rn(nt2, Bi, __ffma2_rn(ns2, Br, __ffma2_rn(c2, Ar, Ar)));
      a.wi[k] = __ffma2_rn(t2, Br, __ffma2_rn(ns2, Bi, __ffma2_rn(c2, Ai, Ai)));
      b.wr[k] = __ffma2_rn(nt2, Ai, __ffma2_rn(s2, Ar, __ffma2_rn(c2, Br, Br)));
      b.wi[k] = __ffma2_rn(t2, Ar, __ffma2_rn(s2, Ai, __ffma2_rn(c2, Bi, Bi)));
    }
  }
}

// Apply a logged rotation (c-1, Re(e s), Im(e s)) to the X planes of a pair (the replay).
template <class C>
__device__ __forceinline__ void apply_rotation(Planes<C>& a, Planes<C>& b, float4 prm) {
  const float2 c2 = f2(prm.x), s2 = f2(prm.y), ns2 = f2(-prm.y), t2 = f2(prm.z), nt2 = f2(-prm.z);
#pragma unroll
  for (int k = 0; k < C::MH; ++k) {
    const float2 Ar = a.xr[k], Ai = a.xi[k], Br = b.xr[k], Bi = b.xi[k];
    a.xr[k] = __ffma2_rn(nt2, Bi, __ffma2_rn(ns2, Br, __ffma2_rn(c2, Ar, Ar)));
    a.xi[k] = __ffma2_rn(t2, Br, __ffma2_rn(ns2, Bi, __ffma2_rn(c2, Ai, Ai)));
    b.xr[k] = __ffma2_rn(nt2, Ai, __ffma2_rn(s2, Ar, __ffma2_rn(c2, Br, Br)));
    b.xi[k] = __ffma2_rn(t2, Ar, __ffma2_rn(s2, Ai, __ffma2_rn(c2, Bi, Bi)));
  }
}

// Write column `a` (id `ida`) to a mailbox slot: lane l stores (re, im) of its row pair k as one
// 16-byte value at k L + l. No barrier inside: the caller may branch around this (team 0 moves a
// different array); the barrier that follows must be reached by every thread in uniform control
// flow (aligned CTA / cluster barriers).
template <class C>
__device__ __forceinline__ void put_column(const Planes<C>& a, int ida, float2* dst, int* dst_id, int lane) {
  constexpr int MH = C::MH, WH = C::WH, L = C::L;
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int k = 0; k < MH; ++k) d[k * L + lane] = make_float4(a.xr[k].x, a.xr[k].y, a.xi[k].x, a.xi[k].y);
  if constexpr (C::VEC) {
    float4* dw = reinterpret_cast<float4*>(dst + C::XR);
#pragma unroll
    for (int k = 0; k < WH; ++k) dw[k * L + lane] = make_float4(a.wr[k].x, a.wr[k].y, a.wi[k].x, a.wi[k].y);
  }
  if (lane == 0) *dst_id = ida;
}

// Read this team's mailbox slot into column `a` (after the barrier).
template <class C>
__device__ __forceinline__ void get_column(Planes<C>& a, int& ida, const float2* src, const int* src_id, int lane) {
  constexpr int MH = C::MH, WH = C::WH, L = C::L;
  const float4* d = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int k = 0; k < MH; ++k) {
    const float4 v = d[k * L + lane];
    a.xr[k] = make_float2(v.x, v.y);
    a.xi[k] = make_float2(v.z, v.w);
  }
  if constexpr (C::VEC) {
    const float4* dw = reinterpret_cast<const float4*>(src + C::XR);
#pragma unroll
    for (int k = 0; k < WH; ++k) {
      const float4 v = dw[k * L + lane];
      a.wr[k] = make_float2(v.x, v.y);
      a.wi[k] = make_float2(v.z, v.w);
    }
  }
  ida = *src_id;
}

// Row slot s (row lane + L s) of the X part / W part as a complex value.
template <class C>
__device__ __forceinline__ float2 x_at(const Planes<C>& a, int s) {
  const int k = s < C::MH ? s : s - C::MH;
  return s < C::MH ? make_float2(a.xr[k].x, a.xi[k].x) : make_float2(a.xr[k].y, a.xi[k].y);
}
template <class C>
__device__ __forceinline__ float2 w_at(const Planes<C>& a, int s) {
  const int k = s < C::WH ? s : s - C::WH;
  return s < C::WH ? make_float2(a.wr[k].x, a.wi[k].x) : make_float2(a.wr[k].y, a.wi[k].y);
}

template <class C, bool FUSED, bool LOG = false>
__global__ void __launch_bounds__(C::BLOCK, C::MINB)
jacobi_kernel(const __grid_constant__ JacobiLaunch P) {
  static_assert(!LOG || (!C::VEC && C::PPT == 1 && C::SPU == 1),
                "the rotation log serves values-mode variants with one symbol per unit");
  constexpr int NP = C::NP, L = C::L, MR = C::MR, WR = C::WR, TC = C::TC, NC = C::NC;
  constexpr int TPC = C::TPC, CS = C::CS, RS = C::RS, PPT = C::PPT;
  constexpr int NCOL = 2 * PPT;   // columns a thread holds rows of
  constexpr int Cn = NC - 1;      // rounds per sweep
  constexpr int FIX = NC - 1;     // the column that stays at position 0
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const int unit = threadIdx.x / C::UT;
  const int ut = threadIdx.x % C::UT;
  const int sym = ut / TC;
  const int st = ut % TC;
  const int lane = st % L;
  int crank = 0;
  if constexpr (CS > 1) crank = (int)cg::this_cluster().block_rank();
  // the thread's teams: PPT consecutive teams of this CTA (local index lteam[j], global team[j])
  int lteam[PPT], team[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    lteam[j] = (st / L) * PPT + j;
    team[j] = crank * TPC + lteam[j];
  }
  unsigned char* ubase = smem_raw + (size_t)unit * C::UNIT_BYTES;
  float2* mbox = reinterpret_cast<float2*>(ubase + (size_t)sym * C::SYM_BYTES);
  float2* phs = mbox + C::MBOX;
  float* ssig = reinterpret_cast<float*>(phs + kMaxTaps);
  int* ubox = reinterpret_cast<int*>(ubase + (size_t)C::SPU * C::SYM_BYTES);  // item, vote[2], zeros
  float* ured = reinterpret_cast<float*>(ubox + 4);                             // UT / 32 floats

  Counters* ctr = P.counters;
  unsigned int* queue = &ctr->queue[P.queue_slot];

  // Mailbox addresses for the two round parities (loop invariant). Position at even rounds
  // is the team index, at odd rounds pi(team); the column a position sends goes to the
  // neighbouring position (0 -> 1, odd -> i-1, even -> i+1), held after the move by team
  // dp (next round odd) or pi(dp) (next round even).
  float2 *dst_e[PPT], *dst_o[PPT];
  int *dst_id_e[PPT], *dst_id_o[PPT];
  const float2 *src_e[PPT], *src_o[PPT];
  const int *src_id_e[PPT], *src_id_o[PPT];
  int* mids = reinterpret_cast<int*>(ssig + NC);   // column ids that travel with the columns
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    auto target = [&](int pos) { return pos == 0 ? 1 : ((pos & 1) ? pos - 1 : pos + 1); };
    const int dest_e = pi_pos<NP>(target(team[j]));        // sent at an even round
    const int dest_o = target(pi_pos<NP>(team[j]));        // sent at an odd round
    dst_e[j] = mbox + (size_t)(0 * TPC + dest_e % TPC) * RS;
    dst_o[j] = mbox + (size_t)(1 * TPC + dest_o % TPC) * RS;
    dst_id_e[j] = mids + 0 * TPC + dest_e % TPC;
    dst_id_o[j] = mids + 1 * TPC + dest_o % TPC;
    if constexpr (CS > 1) {
      cg::cluster_group cl = cg::this_cluster();
      dst_e[j] = cl.map_shared_rank(dst_e[j], dest_e / TPC);
      dst_o[j] = cl.map_shared_rank(dst_o[j], dest_o / TPC);
      dst_id_e[j] = cl.map_shared_rank(dst_id_e[j], dest_e / TPC);
      dst_id_o[j] = cl.map_shared_rank(dst_id_o[j], dest_o / TPC);
    }
    src_e[j] = mbox + (size_t)(0 * TPC + lteam[j]) * RS;
    src_o[j] = mbox + (size_t)(1 * TPC + lteam[j]) * RS;
    src_id_e[j] = mids + 0 * TPC + lteam[j];
    src_id_o[j] = mids + 1 * TPC + lteam[j];
  }

  for (;;) {
    // ---------------------------------------------------------------- fetch a work item
    int item;
    if constexpr (CS > 1) {
      cg::cluster_group cl = cg::this_cluster();
      if (crank == 0 && threadIdx.x == 0) {
        const int it = (int)atomicAdd(queue, 1u);
        for (int r = 0; r < CS; ++r) *cl.map_shared_rank(&ubox[0], r) = it;
        ubox[1] = 0;
        ubox[2] = 0;
      }
      cl.sync();
      item = ubox[0];
    } else if constexpr (C::UT == 32) {
      int v = 0;
      if (ut == 0) v = (int)atomicAdd(queue, 1u);
      item = __shfl_sync(0xffffffffu, v, 0);
    } else {
      if (ut == 0) ubox[0] = (int)atomicAdd(queue, 1u);
      __syncthreads();
      item = ubox[0];
      __syncthreads();
    }
    if (item >= P.total_items) break;
    int li = 0;
    while (li + 1 < P.nlayers && item >= P.L[li + 1].item_begin) ++li;
    const LayerArgs& La = P.L[li];
    const int h = (item - La.item_begin) * C::SPU + sym;
    const bool active = h < La.F_h;
    const int kk = La.kh * La.kw;
    const int f = active ? La.half[h] : 0;
    const int jj = f / La.m;
    const int ll = f - jj * La.m;
    const int N = La.N, M = La.M;

    // ---------------------------------------------------------------- phases exp(2 pi i <k, q_ab>)
    // q_ab = floor(y_ab / s): the tap's coarse offset (q = y at stride 1)
    if constexpr (FUSED) {
      for (int t = st; t < kk; t += TC) {
        const int a = t / La.kw, b = t - a * La.kw;
        phs[t] = tap_phase(La, jj, ll, a, b);
      }
      unit_sync<C>();
    }

    // ---------------------------------------------------------------- round-0 pair of each team
    // Two register arrays per team. Every team except team 0 keeps its newest column and
    // sends its older one, so at round t the column that moves is the one in array (t & 1):
    // arrays alternate by round parity and the moving array is static in the 2-way unrolled
    // loop. Team 0 keeps the fixed column NC-1 in array 0 and moves array 1 every round.
    // Round 0: position k holds (c(k), c(-k)), or (c(0), NC-1) for k = 0; the column that
    // leaves first goes to array 0 (array 1 for team 0).
    int id0[PPT], id1[PPT];
    Planes<C> c0[PPT], c1[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int tm = team[j];
      if (tm == 0) { id0[j] = FIX; id1[j] = 0; }
      else if ((tm & 1) || tm == NP - 1) { id0[j] = tm; id1[j] = Cn - tm; }
      else { id0[j] = Cn - tm; id1[j] = tm; }
#pragma unroll
      for (int k = 0; k < C::MH; ++k) {
        const int r0 = lane + L * k, r1 = lane + L * (k + C::MH);
        const float2 a0 = active ? x_entry<FUSED>(La, h, r0, id0[j], phs) : make_float2(0.f, 0.f);
        const float2 a1 = active ? x_entry<FUSED>(La, h, r1, id0[j], phs) : make_float2(0.f, 0.f);
        const float2 b0 = active ? x_entry<FUSED>(La, h, r0, id1[j], phs) : make_float2(0.f, 0.f);
        const float2 b1 = active ? x_entry<FUSED>(La, h, r1, id1[j], phs) : make_float2(0.f, 0.f);
        c0[j].xr[k] = make_float2(a0.x, a1.x);
        c0[j].xi[k] = make_float2(a0.y, a1.y);
        c1[j].xr[k] = make_float2(b0.x, b1.x);
        c1[j].xi[k] = make_float2(b0.y, b1.y);
      }
      if constexpr (C::VEC) {
        // W starts as the identity; rows beyond WR per lane are padding and stay zero
#pragma unroll
        for (int k = 0; k < C::WH; ++k) {
          const int r0 = lane + L * k, r1 = lane + L * (k + C::WH);
          const bool v1 = k + C::WH < WR;
          c0[j].wr[k] = make_float2(r0 == id0[j] && r0 < N ? 1.f : 0.f, v1 && r1 == id0[j] && r1 < N ? 1.f : 0.f);
          c1[j].wr[k] = make_float2(r0 == id1[j] && r0 < N ? 1.f : 0.f, v1 && r1 == id1[j] && r1 < N ? 1.f : 0.f);
          c0[j].wi[k] = make_float2(0.f, 0.f);
          c1[j].wi[k] = make_float2(0.f, 0.f);
        }
      }
    }

    // ---------------------------------------------------------------- sweeps
    const float tol2 = La.tol2;
    int sweeps = 0, nrot = 0, rr = 0, rotated = 0;
    bool converged = false;
    int t = 0;       // round counter (rotation log)
    int t_rot = 0;   // rounds up to the end of the last sweep in which this symbol rotated
    // a sweep ends every Cn rounds; returns true when the unit stops
    auto sweep_end = [&]() -> bool {
      rr = 0;
      ++sweeps;
      bool any_sym, any_unit;
      if constexpr (CS > 1) {
        cg::cluster_group cl = cg::this_cluster();
        const int q = sweeps & 1;
        const int mine = __syncthreads_or(rotated);
        if (threadIdx.x == 0 && mine) atomicOr(cl.map_shared_rank(&ubox[1 + q], 0), 1);
        cl.sync();
        any_unit = *cl.map_shared_rank(&ubox[1 + q], 0) != 0;
        if (crank == 0 && threadIdx.x == 0) ubox[2 - q] = 0;   // the other parity, used next sweep
        any_sym = any_unit;
      } else if constexpr (C::UT == 32) {
        const unsigned bal = __ballot_sync(0xffffffffu, rotated != 0);
        any_sym = (bal & sym_mask<TC>(sym)) != 0u;
        any_unit = bal != 0u;
      } else {
        any_unit = __syncthreads_or(rotated) != 0;
        any_sym = any_unit;
      }
      rotated = 0;
      if (any_sym) t_rot = t;
      if (!any_sym && !converged) {
        converged = true;
        if (st == 0 && crank == 0 && active) atomicAdd(&ctr->sweeps, (unsigned long long)sweeps);
      }
      return !any_unit || sweeps >= P.max_sweeps;
    };
    float4* lg = nullptr;
    if constexpr (LOG) lg = P.log + (size_t)h * P.log_cap * NP + team[0];
    // One round on every pair of the thread: all dot products first, then all rotation
    // parameters (independent chains the scheduler can interleave), then the rotations.
    auto round = [&]() {
      float al[PPT], be[PPT], gr[PPT], gi[PPT];
      bool rot[PPT];
      bool any = false;
#pragma unroll
      for (int j = 0; j < PPT; ++j) pair_dots<C>(c0[j], c1[j], al[j], be[j], gr[j], gi[j]);
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        rot[j] = pair_test(al[j], be[j], gr[j], gi[j], tol2);
        any = any || rot[j];
      }
      float4 prm[PPT];
      if (any) {
#pragma unroll
        for (int j = 0; j < PPT; ++j) prm[j] = pair_params(al[j], be[j], gr[j], gi[j], rot[j]);
#pragma unroll
        for (int j = 0; j < PPT; ++j)
          if (rot[j]) {
            rotate_pair<C>(c0[j], c1[j], prm[j]);
            rotated = 1;
            ++nrot;
          }
      }
      if constexpr (LOG) {
        if (lane == 0 && active && t < P.log_cap)
          lg[(size_t)t * NP] = rot[0] ? prm[0] : make_float4(0.f, 0.f, 0.f, 0.f);
        ++t;
      }
    };
    for (;;) {
      // even round: teams move array 0, team 0 moves array 1
      round();
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        if (team[j] == 0) put_column<C>(c1[j], id1[j], dst_e[j], dst_id_e[j], lane);
        else put_column<C>(c0[j], id0[j], dst_e[j], dst_id_e[j], lane);
      }
      sym_sync<C>();
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        if (team[j] == 0) get_column<C>(c1[j], id1[j], src_e[j], src_id_e[j], lane);
        else get_column<C>(c0[j], id0[j], src_e[j], src_id_e[j], lane);
      }
      if (++rr == Cn && sweep_end()) break;
      // odd round: every team moves array 1
      round();
#pragma unroll
      for (int j = 0; j < PPT; ++j) put_column<C>(c1[j], id1[j], dst_o[j], dst_id_o[j], lane);
      sym_sync<C>();
#pragma unroll
      for (int j = 0; j < PPT; ++j) get_column<C>(c1[j], id1[j], src_o[j], src_id_o[j], lane);
      if (++rr == Cn && sweep_end()) break;
    }
    if (!converged && st == 0 && crank == 0 && active) {
      atomicAdd(&ctr->sweeps, (unsigned long long)sweeps);
      atomicAdd(&ctr->unconverged, 1ull);
    }
    if (lane == 0 && nrot && active) atomicAdd(&ctr->rotations, (unsigned long long)nrot);
    if constexpr (LOG) {
      // raw X columns in column order; sigma, order and vectors come from the finalize kernel.
      // The replay stops after the last sweep that rotated: later rounds only move columns,
      // and W is written by column id.
      if (st == 0 && crank == 0 && active) P.rounds[h] = t_rot < P.log_cap ? t_rot : P.log_cap;
      if (active) {
        float2* xo = P.xraw + (size_t)h * M * N;
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const int row = lane + L * i;
          if (row < M) {
            if (id0[0] < N) xo[(size_t)row * N + id0[0]] = x_at<C>(c0[0], i);
            if (id1[0] < N) xo[(size_t)row * N + id1[0]] = x_at<C>(c1[0], i);
          }
        }
      }
      sym_sync<C>();
      continue;
    }

    // ---------------------------------------------------------------- singular values, order
    // the thread's columns: 2 j (array 0 of team j) and 2 j + 1 (array 1)
    auto col = [&](int kc) -> Planes<C>& { return (kc & 1) ? c1[kc >> 1] : c0[kc >> 1]; };
    int cid[NCOL];
    float al[NCOL], sg[NCOL], nw[NCOL];
#pragma unroll
    for (int kc = 0; kc < NCOL; ++kc) {
      cid[kc] = (kc & 1) ? id1[kc >> 1] : id0[kc >> 1];
      const Planes<C>& X = col(kc);
      float a = 0.f;
#pragma unroll
      for (int i = 0; i < MR; ++i) {
        const float2 x = x_at<C>(X, i);
        a = fmaf(x.x, x.x, fmaf(x.y, x.y, a));
      }
      al[kc] = team_sum<L>(a);
      sg[kc] = sqrtf(al[kc]);
      nw[kc] = 1.f;   // norm of the accumulated rotation column (1 up to rounding)
      if constexpr (C::VEC) {
        float q = 0.f;
#pragma unroll
        for (int i = 0; i < WR; ++i) {
          const float2 w = w_at<C>(X, i);
          q = fmaf(w.x, w.x, fmaf(w.y, w.y, q));
        }
        q = team_sum<L>(q);
        // x_p = A w_p up to rounding, so sigma_p = |x_p| / |w_p| with v_p = w_p / |w_p|
        nw[kc] = q > 0.f ? sqrtf(q) : 1.f;
        sg[kc] = sg[kc] / nw[kc];
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int kc = 0; kc < NCOL; ++kc) {
        if (cid[kc] >= N) continue;
        if constexpr (CS > 1) {
          cg::cluster_group cl = cg::this_cluster();
          for (int r = 0; r < CS; ++r) cl.map_shared_rank(ssig, r)[cid[kc]] = sg[kc];
        } else {
          ssig[cid[kc]] = sg[kc];
        }
      }
    }
    sym_sync<C>();
    int rk[NCOL];
#pragma unroll
    for (int kc = 0; kc < NCOL; ++kc) rk[kc] = 0;
    bool finite = true;
    float smax = 0.f;
    for (int q = 0; q < N; ++q) {
      const float v = ssig[q];
      finite = finite && isfinite(v);
      smax = fmaxf(smax, v);
#pragma unroll
      for (int kc = 0; kc < NCOL; ++kc) rk[kc] += (v > sg[kc]) || (v == sg[kc] && q < cid[kc]);
    }
    if (active && st == 0 && crank == 0 && !finite) atomicAdd(&ctr->nonfinite, 1ull);
    if (active && lane == 0) {
      const int r = La.r;
      float* row = La.sigma + (size_t)(P.half_output ? h : f) * r;
      const int fc = ((La.n - jj) % La.n) * La.m + (La.m - ll) % La.m;
      float* rowc = (!P.half_output && fc != f) ? La.sigma + (size_t)fc * r : nullptr;
#pragma unroll
      for (int kc = 0; kc < NCOL; ++kc) {
        if (cid[kc] >= N) continue;
        row[rk[kc]] = sg[kc];
        if (rowc) rowc[rk[kc]] = sg[kc];
      }
    }

    if constexpr (C::VEC) {
      // A column far below sigma_max (or whose squared norm is below 2^-100, the bound under
      // which the sweeps leave pairs unrotated) carries no direction: treat it as a zero
      // singular value (or NaN) and complete it below.
      bool zc[NCOL];
      float ix[NCOL], iw[NCOL];
#pragma unroll
      for (int kc = 0; kc < NCOL; ++kc) {
        zc[kc] = !(sg[kc] > 1e-12f * smax) || !(al[kc] > 0x1p-100f);
        ix[kc] = zc[kc] ? 0.f : __frsqrt_rn(al[kc]);
        iw[kc] = 1.f / nw[kc];
      }
      float2* Xo = La.wide ? La.V : La.U;     // normalised X columns
      float2* Wo = La.wide ? La.U : La.V;     // accumulated rotations
      if constexpr (CS > 1) {
        // columns are spread over the cluster: write them straight to their rank in HBM
        if (active) {
          float2* xo = Xo + (size_t)h * M * N;
          float2* wo = Wo + (size_t)h * N * N;
#pragma unroll
          for (int kc = 0; kc < NCOL; ++kc) {
            if (cid[kc] >= N) continue;
            if (!LFA_DOK(La.dbg, rk[kc] >= 0 && rk[kc] < N && h < La.F_h, 1)) continue;   // cluster output: rank
            const Planes<C>& X = col(kc);
#pragma unroll
            for (int i = 0; i < MR; ++i) {
              const int row = lane + L * i;
              const float2 x = x_at<C>(X, i);
              if (row < M) xo[(size_t)row * N + rk[kc]] = make_float2(x.x * ix[kc], x.y * ix[kc]);
            }
#pragma unroll
            for (int i = 0; i < WR; ++i) {
              const int row = lane + L * i;
              const float2 w = w_at<C>(X, i);
              if (row < N) wo[(size_t)row * N + rk[kc]] = make_float2(w.x * iw[kc], w.y * iw[kc]);
            }
          }
        }
      } else {
        // ------------------------------------------------------------ stage U / V by rank
        // mailbox column `rank`: normalised X rows [0, XR), W rows [XR, XR + WRC)
        constexpr int CSx = C::XR + C::WRC;
        int* defc = ubox + 3;
        if (ut == 0) *defc = 0;
        unit_sync<C>();
#pragma unroll
        for (int kc = 0; kc < NCOL; ++kc) {
          if (cid[kc] >= N) continue;
          if (!LFA_DOK(La.dbg, rk[kc] >= 0 && rk[kc] < N, 2)) continue;   // staged output: rank
          const Planes<C>& X = col(kc);
          float2* d = mbox + (size_t)rk[kc] * CSx;
#pragma unroll
          for (int i = 0; i < MR; ++i) {
            const float2 x = x_at<C>(X, i);
            d[lane + L * i] = make_float2(x.x * ix[kc], x.y * ix[kc]);
          }
#pragma unroll
          for (int i = 0; i < WR; ++i) {
            const float2 w = w_at<C>(X, i);
            d[C::XR + lane + L * i] = make_float2(w.x * iw[kc], w.y * iw[kc]);
          }
          if (zc[kc] && lane == 0) { ssig[cid[kc]] = -1.f; atomicAdd(defc, 1); }
        }
        unit_sync<C>();
        // ------------------------------------------------------------ complete zero columns
        // A zero singular value leaves x_p = 0; its left vector is any unit vector orthogonal
        // to the others: Gram-Schmidt of the canonical vectors e_k against the accepted columns
        // (the ranks before it), in rank order.
        if (*defc > 0) {
          for (int sidx = 0; sidx < C::SPU; ++sidx) {
            float2* mb = reinterpret_cast<float2*>(ubase + (size_t)sidx * C::SYM_BYTES);
            const float* sg = reinterpret_cast<const float*>(mb + C::MBOX + kMaxTaps);
            float2* tmp = mb + C::MBOX;  // the phase grid is no longer needed
            const int hh = (item - La.item_begin) * C::SPU + sidx;
            if (hh >= La.F_h) continue;
            int zc = 0;
            for (int q = 0; q < N; ++q) zc += (sg[q] == -1.f);
            int kstart = 0;
            for (int d = N - zc; d < N; ++d) {
              for (int k = kstart; k < M; ++k) {
                float nrm = 0.f;
                for (int row = ut; row < M; row += C::UT) {
                  float vr = (row == k) ? 1.f : 0.f, vi = 0.f;
                  for (int q = 0; q < d; ++q) {
                    const float2 uq = mb[(size_t)q * CSx + row];
                    const float2 uk = mb[(size_t)q * CSx + k];
                    vr -= uq.x * uk.x + uq.y * uk.y;   // v -= u_q conj(u_q[k])
                    vi -= uq.y * uk.x - uq.x * uk.y;
                  }
                  tmp[row] = make_float2(vr, vi);
                  nrm += vr * vr + vi * vi;
                }
                nrm = unit_sum<C>(nrm, ured);
                if (nrm > 0.25f) {
                  const float inv = __frsqrt_rn(nrm);
                  for (int row = ut; row < M; row += C::UT)
                    mb[(size_t)d * CSx + row] = make_float2(tmp[row].x * inv, tmp[row].y * inv);
                  kstart = k + 1;
                  unit_sync<C>();
                  break;
                }
                unit_sync<C>();
              }
            }
          }
          unit_sync<C>();
        }
        // ------------------------------------------------------------ coalesced write-out
        if (active) {
          float2* xo = Xo + (size_t)h * M * N;
          for (int e = st; e < M * N; e += TC) {
            const int row = e / N, s = e - row * N;
            xo[e] = mbox[(size_t)s * CSx + row];
          }
          float2* wo = Wo + (size_t)h * N * N;
          for (int e = st; e < N * N; e += TC) {
            const int row = e / N, s = e - row * N;
            wo[e] = mbox[(size_t)s * CSx + C::XR + row];
          }
        }
      }
    }
    sym_sync<C>();
  }
  if constexpr (CS > 1) cg::this_cluster().sync();   // no CTA leaves while others may address it
}

}  // namespace lfa
