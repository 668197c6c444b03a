// Replay of a rotation log onto W = I: the right (or, for wide symbols, left) singular
// vectors of symbols whose accumulated rotation matrix W does not fit in registers next to X
// (512 columns), or whose forward is faster without carrying W (the autotuner's choice). The forward kernel ran in values mode and logged, per round and team, the
// rotation it applied; rotations act on columns, so the rows of W are independent and can be
// rebuilt in row blocks by one CTA each, following the same round-robin schedule (the same
// team movement and exchange as the forward kernel) with the logged parameters.
#include "jacobi.cuh"

namespace lfa {

template <class C>
__global__ void __launch_bounds__(C::TC) replay_kernel(const __grid_constant__ ReplayArgs R) {
  constexpr int NP = C::NP, L = C::L, MR = C::MR, NC = C::NC, TPC = C::TPC, RS = C::RS;
  constexpr int Cn = NC - 1, FIX = NC - 1, RB = C::XR;
  static_assert(C::CS == 1 && !C::VEC, "the replay runs one CTA per row block");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* mbox = reinterpret_cast<float2*>(smem_raw);
  int* mids = reinterpret_cast<int*>(mbox + C::MBOX);

  const int team = threadIdx.x / L;
  const int lane = threadIdx.x % L;
  const int slot = blockIdx.y;
  const int row0 = blockIdx.x * RB;
  const int N = R.La.N;

  // mailbox addresses, as in the forward kernel
  auto target = [&](int pos) { return pos == 0 ? 1 : ((pos & 1) ? pos - 1 : pos + 1); };
  const int dest_e = pi_pos<NP>(target(team));
  const int dest_o = target(pi_pos<NP>(team));
  float2* dst_e = mbox + (size_t)(0 * TPC + dest_e) * RS;
  float2* dst_o = mbox + (size_t)(1 * TPC + dest_o) * RS;
  int* dst_id_e = mids + 0 * TPC + dest_e;
  int* dst_id_o = mids + 1 * TPC + dest_o;
  const float2* src_e = mbox + (size_t)(0 * TPC + team) * RS;
  const float2* src_o = mbox + (size_t)(1 * TPC + team) * RS;
  const int* src_id_e = mids + 0 * TPC + team;
  const int* src_id_o = mids + 1 * TPC + team;

  // round-0 columns of this team (see the forward kernel) and W = I restricted to the block
  int id0, id1;
  if (team == 0) { id0 = FIX; id1 = 0; }
  else if ((team & 1) || team == NP - 1) { id0 = team; id1 = Cn - team; }
  else { id0 = Cn - team; id1 = team; }
  Planes<C> c0, c1;
#pragma unroll
  for (int k = 0; k < C::MH; ++k) {
    const int r0 = row0 + lane + L * k, r1 = row0 + lane + L * (k + C::MH);
    c0.xr[k] = make_float2(r0 == id0 && r0 < N ? 1.f : 0.f, r1 == id0 && r1 < N ? 1.f : 0.f);
    c1.xr[k] = make_float2(r0 == id1 && r0 < N ? 1.f : 0.f, r1 == id1 && r1 < N ? 1.f : 0.f);
    c0.xi[k] = make_float2(0.f, 0.f);
    c1.xi[k] = make_float2(0.f, 0.f);
  }

  const int T = R.rounds[slot];
  const float4* lg = R.log + (size_t)slot * R.log_cap * NP + team;
  // The log is read four rounds ahead (the rounds themselves have no other long-latency step).
  // T is the same for every thread, so every break below is uniform and the barriers stay aligned.
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 cur[4], nxt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) cur[k] = k < T ? __ldg(lg + (size_t)k * NP) : zero;
  auto rotate = [&](const float4& e) {
    if (e.x != 0.f || e.y != 0.f || e.z != 0.f) apply_rotation<C>(c0, c1, e);
  };
  for (int t = 0; t < T; t += 4) {
#pragma unroll
    for (int k = 0; k < 4; ++k) nxt[k] = t + 4 + k < T ? __ldg(lg + (size_t)(t + 4 + k) * NP) : zero;
    // rounds t and t + 2 are even (teams move array 0, team 0 moves array 1), t + 1 and t + 3 odd
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
      if (t + k >= T) break;
      rotate(cur[k]);
      if (team == 0) put_column<C>(c1, id1, dst_e, dst_id_e, lane);
      else put_column<C>(c0, id0, dst_e, dst_id_e, lane);
      __syncthreads();
      if (team == 0) get_column<C>(c1, id1, src_e, src_id_e, lane);
      else get_column<C>(c0, id0, src_e, src_id_e, lane);
      if (t + k + 1 >= T) break;
      rotate(cur[k + 1]);
      put_column<C>(c1, id1, dst_o, dst_id_o, lane);
      __syncthreads();
      get_column<C>(c1, id1, src_o, src_id_o, lane);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
  }

  // the block's rows of the team's two columns, in column order
  float2* W = R.wraw + (size_t)slot * N * N;
#pragma unroll
  for (int i = 0; i < MR; ++i) {
    const int row = row0 + lane + L * i;
    if (row < N) {
      if (id0 < N) W[(size_t)row * N + id0] = x_at<C>(c0, i);
      if (id1 < N) W[(size_t)row * N + id1] = x_at<C>(c1, i);
    }
  }
}

// Finalize one symbol: x_c = A w_c up to rounding for every column c, so sigma_c = |x_c| / |w_c|
// with u_c = x_c / |x_c| and v_c = w_c / |w_c| (the roles swap for wide symbols); the columns
// are ranked by descending sigma (ties by column index) and written in that order. One CTA
// per symbol, one thread per column; fixed-order sums (deterministic).
__global__ void __launch_bounds__(512) finalize_kernel(const __grid_constant__ ReplayArgs R) {
  __shared__ float sg[512];
  const LayerArgs& La = R.La;
  const int slot = blockIdx.x;
  const int c = threadIdx.x;
  const int M = La.M, N = La.N;
  const float2* X = R.xraw + (size_t)slot * M * N;
  const float2* Wr = R.wraw + (size_t)slot * N * N;
  float xn = 0.f, wn = 0.f;
  if (c < N) {
    for (int row = 0; row < M; ++row) {
      const float2 v = X[(size_t)row * N + c];
      xn = fmaf(v.x, v.x, fmaf(v.y, v.y, xn));
    }
    for (int row = 0; row < N; ++row) {
      const float2 v = Wr[(size_t)row * N + c];
      wn = fmaf(v.x, v.x, fmaf(v.y, v.y, wn));
    }
  }
  const float ixn = xn > 0x1p-100f ? rsqrt_nr(xn) : 0.f;   // zero-column bound of the sweeps
  const float iwn = wn > 0.f ? rsqrt_nr(wn) : 0.f;
  const float sc = xn * ixn * iwn;   // |x| / |w|
  if (c < N) sg[c] = sc;
  __syncthreads();
  int rank = 0;
  bool finite = true;
  float smax = 0.f;
  if (c < N) {
    for (int q = 0; q < N; ++q) {
      const float v = sg[q];
      finite = finite && isfinite(v);
      smax = fmaxf(smax, v);
      rank += (v > sc) || (v == sc && q < c);
    }
  }
  // a column far below sigma_max carries no direction: write it as zero (completed afterwards)
  const float ixz = sc > 1e-12f * smax ? ixn : 0.f;
  if (__syncthreads_or(c < N && !finite) && c == 0) atomicAdd(&R.counters->nonfinite, 1ull);
  if (c >= N) return;
  const int h = slot;
  const int f = La.half[h];
  const int jj = f / La.m, ll = f - jj * La.m;
  const int r = La.r;
  float* row = La.sigma + (size_t)(R.half_output ? h : f) * r;
  if (!LFA_DOK(La.dbg, rank >= 0 && rank < N && h < La.F_h, 4)) return;   // finalize: rank, symbol
  row[rank] = sc;
  if (!R.half_output) {
    const int fc = ((La.n - jj) % La.n) * La.m + (La.m - ll) % La.m;
    if (fc != f) La.sigma[(size_t)fc * r + rank] = sc;
  }
  float2* Xo = (La.wide ? La.V : La.U) + (size_t)h * M * N;
  float2* Wo = (La.wide ? La.U : La.V) + (size_t)h * N * N;
  for (int rw = 0; rw < M; ++rw) {
    const float2 v = X[(size_t)rw * N + c];
    Xo[(size_t)rw * N + rank] = make_float2(v.x * ixz, v.y * ixz);
  }
  for (int rw = 0; rw < N; ++rw) {
    const float2 v = Wr[(size_t)rw * N + c];
    Wo[(size_t)rw * N + rank] = make_float2(v.x * iwn, v.y * iwn);
  }
}

// Row blocks of XR = MR L = 32 rows: 16 rows of each of the team's two columns per lane on two
// lanes per pair (four lanes of 8 rows for 16 pairs; one lane of 32 rows for 32 pairs, a one-warp
// CTA whose barrier is a warp's), so that every replay CTA has at least 32 threads, one unit.
// (16-row blocks for 32 pairs were slower: every block re-reads the symbol's log.)
using ReplayC256 = JCfg<256, 2, 16, 1, false, 1>;
using ReplayC128 = JCfg<128, 2, 16, 1, false, 1>;
using ReplayC64 = JCfg<64, 2, 16, 1, false, 1>;
using ReplayC32 = JCfg<32, 1, 32, 1, false, 1>;   // one lane per team, 32 rows: a one-warp CTA
using ReplayC16 = JCfg<16, 4, 8, 1, false, 1>;
static_assert(ReplayC16::SPU == 1 && ReplayC32::SPU == 1, "one symbol per replay CTA");

// A replay CTA holds one symbol's row block: TC threads and one unit of shared memory (a
// configuration whose unit is a single warp would otherwise be launched as four units).
template <class C>
constexpr size_t replay_smem() { return C::SYM_BYTES + C::TAIL_BYTES; }

template <class C>
static cudaError_t replay_t(const ReplayArgs& R, int symbols, cudaStream_t s) {
  cudaError_t e;
  const int N = R.La.N;
  dim3 grid((unsigned)((N + C::XR - 1) / C::XR), (unsigned)symbols);
  replay_kernel<C><<<grid, C::TC, replay_smem<C>(), s>>>(R);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<<<symbols, 512, 0, s>>>(R);
  return cudaGetLastError();
}

template <class C>
static cudaError_t prepare_t() {
  return cudaFuncSetAttribute(replay_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)replay_smem<C>());
}

bool replay_supported(int NP) { return NP == 16 || NP == 32 || NP == 64 || NP == 128 || NP == 256; }

cudaError_t prepare_replay(int NP) {
  switch (NP) {
    case 256: return prepare_t<ReplayC256>();
    case 128: return prepare_t<ReplayC128>();
    case 64: return prepare_t<ReplayC64>();
    case 32: return prepare_t<ReplayC32>();
    case 16: return prepare_t<ReplayC16>();
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_replay(int NP, const ReplayArgs& R, int symbols, cudaStream_t s, int* nkernels) {
  *nkernels = 2;
  if (symbols <= 0) return cudaSuccess;
  if (symbols > 65535 || R.La.N > 512) return cudaErrorInvalidValue;
  switch (NP) {
    case 256: return replay_t<ReplayC256>(R, symbols, s);
    case 128: return replay_t<ReplayC128>(R, symbols, s);
    case 64: return replay_t<ReplayC64>(R, symbols, s);
    case 32: return replay_t<ReplayC32>(R, symbols, s);
    case 16: return replay_t<ReplayC16>(R, symbols, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lfa
