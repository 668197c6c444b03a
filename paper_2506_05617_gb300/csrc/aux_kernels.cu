// Auxiliary kernels of the LFA SVD library (arXiv 2506.05617, Sec. III; strided layers as
// crystals):
//  * symbol assembly into memory (the plain path and lfa_symbols),
//  * lifting of symbol singular vectors to global singular vectors,
//  * the backward pass dL/dw,
//  * the spectral regulariser's dL/dsigma.
#include "half_grid.cuh"
#include "lfa_internal.cuh"

namespace lfa {

__device__ __forceinline__ int mod_pos(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ----------------------------------------------------------------------------- symbols
// A_k[o][i] = sum_{a,b} w[o,i,a,b] exp(2 pi i <k, q_ab>) for the half-grid frequencies (symbol
// definition, Sec. III; for a stride, column i = (ci, u) sums the taps congruent to u). One CTA
// per frequency; the kh x kw phase grid is built once in shared memory; threads stride over
// the symbol's (o, i) entries.
__global__ void __launch_bounds__(256) symbols_kernel(LayerArgs La, float2* out) {
  __shared__ float2 phs[kMaxTaps];
  const int h = blockIdx.x;
  const int f = La.half[h];
  const int j = f / La.m, l = f - j * La.m;
  const int kk = La.kh * La.kw;
  for (int t = threadIdx.x; t < kk; t += blockDim.x) {
    const int a = t / La.kw, b = t - a * La.kw;
    phs[t] = tap_phase(La, j, l, a, b);
  }
  __syncthreads();
  const int CC = La.c_out * La.c_in;
  float2* o = out + (size_t)h * CC;
  for (int e = threadIdx.x; e < CC; e += blockDim.x) {
    const int oo = e / La.c_in, i = e - oo * La.c_in;
    o[e] = symbol_entry(La, oo, i, phs);
  }
}

// Stride-1 layers with at most KK taps: one thread per symbol entry (o, i) keeps the entry's taps in
// registers and writes the entry for a block of SB frequencies, whose k_h x k_w phase grids are
// staged in shared memory; the weights are then read once per SB symbols instead of once per
// symbol, and each frequency's row of entries is written coalesced (consecutive i per warp).
constexpr int kSymbolsBlock = 16;
template <int KK>
__global__ void __launch_bounds__(256) symbols_tiled_kernel(LayerArgs La, float2* out) {
  __shared__ float2 phs[kSymbolsBlock][KK];
  const int kk = La.kh * La.kw;
  const int h0 = blockIdx.y * kSymbolsBlock;
  const int nh = min(kSymbolsBlock, La.F_h - h0);
  for (int x = threadIdx.x; x < nh * kk; x += blockDim.x) {
    const int hh = x / kk, t = x - hh * kk;
    const int f = La.half[h0 + hh];
    const int j = f / La.m, l = f - j * La.m;
    phs[hh][t] = tap_phase(La, j, l, t / La.kw, t % La.kw);
  }
  __syncthreads();
  const int CC = La.c_out * La.c_in;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= CC) return;
  float wt[KK];
  const float* wp = La.w + (size_t)e * kk;   // stride 1: entry (o, i) is weight row o * c_in + i
#pragma unroll
  for (int t = 0; t < KK; ++t) wt[t] = t < kk ? __ldg(wp + t) : 0.f;
  for (int hh = 0; hh < nh; ++hh) {
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int t = 0; t < KK; ++t) {
      if (t < kk) {
        const float2 p = phs[hh][t];
        re = fmaf(wt[t], p.x, re);
        im = fmaf(wt[t], p.y, im);
      }
    }
    out[(size_t)(h0 + hh) * CC + e] = make_float2(re, im);
  }
}

cudaError_t launch_symbols(const LayerArgs& La, float2* out, cudaStream_t s) {
  if (La.F_h <= 0) return cudaSuccess;
  const int kk = La.kh * La.kw;
  if (La.sh == 1 && La.sw == 1 && kk <= 25) {
    const int CC = La.c_out * La.c_in;
    dim3 grid((unsigned)((CC + 255) / 256), (unsigned)((La.F_h + kSymbolsBlock - 1) / kSymbolsBlock));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    if (kk <= 1) symbols_tiled_kernel<1><<<grid, 256, 0, s>>>(La, out);
    else if (kk <= 9) symbols_tiled_kernel<9><<<grid, 256, 0, s>>>(La, out);
    else symbols_tiled_kernel<25><<<grid, 256, 0, s>>>(La, out);
    return cudaGetLastError();
  }
  symbols_kernel<<<La.F_h, 256, 0, s>>>(La, out);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- expansion
// u_hat[q][c][x1][x2] = U_f[c][s] exp(2 pi i (j x1/n + l x2/m)) / sqrt(nm), q = f*r + s
// (U^_k = F_k U_k, Sec. III). U_f = U[h] on the half grid, conj(U[h(fc)]) otherwise.
// For a stride, v_hat lives on the fine torus: v_hat[q][ci][sh x1 + uh][sw x2 + uw] takes
// row (ci, uh, uw) of V_f with the coarse mode of (x1, x2).
//
// A warp serves one output row (vector channel c, grid row z1) for a group of kExpandVecs
// consecutive vectors q (blockIdx.y). Lane i works out vector q0 + i's frequency, half-grid position
// (a closed form), row phase and scaled source entry, all lanes at once (one load each, in
// parallel); the warp then writes the row of each vector in turn, coalesced, taking that vector's
// values from lane i by shuffles. Phase indices are exact 32-bit products mod n or m (j, x1 < n <=
// 65536, so j x1 < 2^32); along a stride-1 row the column index advances by 32 l mod m per step.
constexpr int kExpandRowsPerCTA = 8;   // one row per warp
constexpr int kExpandVecs = 32;

__global__ void __launch_bounds__(256) expand_kernel(LayerArgs La, const float2* U, const float2* V,
                                                     int64_t first, int64_t count, float2* u_hat,
                                                     float2* v_hat) {
  const int n = La.n, m = La.m, r = La.r;
  const float scale = rsqrtf((float)n * (float)m);
  const int lane = threadIdx.x & 31;
  // rows per vector: c_out n + c_w sh n <= 512 * 65536 * 8 < 2^31
  const int rows_u = u_hat ? La.c_out * n : 0;
  const int rows_v = v_hat ? La.c_w * La.sh * n : 0;   // input channels x fine rows
  const int R = blockIdx.x * kExpandRowsPerCTA + (threadIdx.x >> 5);
  if (R >= rows_u + rows_v) return;                    // whole warps; no barriers below
  const bool upart = R < rows_u;
  const int row = upart ? R : R - rows_u;
  const int sh = upart ? 1 : La.sh, sw = upart ? 1 : La.sw;
  const int C = upart ? La.c_out : La.c_in;            // rows of the source factor
  const float2* Src = upart ? U : V;
  float2* dst = upart ? u_hat : v_hat;
  // row -> (channel ci of the output grid, fine row z1); the output grid is (sh n) x (sw m)
  const int fine_rows = sh * n;
  const int ci = row / fine_rows;
  const int z1 = row - ci * fine_rows;
  const int x1 = z1 / sh, uh = z1 - x1 * sh;
  const int len = sw * m;
  const size_t row_off = ((size_t)ci * fine_rows + z1) * len;
  const int src_row = (ci * sh + uh) * sw;              // + u_w along a strided row
  const int64_t q0 = first + (int64_t)blockIdx.y * kExpandVecs;
  const int nv = (int)(first + count - q0 < kExpandVecs ? first + count - q0 : kExpandVecs);
  // lane i < nv: vector q0 + i
  float2 my_a = make_float2(0.f, 0.f), my_pa = make_float2(0.f, 0.f);
  unsigned my_l = 0;
  int my_conj = 0;
  int64_t my_src = 0;
  if (lane < nv) {
    const int64_t q = q0 + lane;
    const int f = (int)(q / r), sv = (int)(q - (int64_t)f * r);
    const unsigned j = (unsigned)(f / m);
    my_l = (unsigned)(f - (int)j * m);
    const int fc = ((n - (int)j) % n) * m + (m - (int)my_l) % m;
    my_conj = fc < f;
    my_pa = La.tw_n[(j * (unsigned)x1) % (unsigned)n];
    const int64_t hp = half_position(n, m, f);
    my_src = LFA_DOK(La.dbg, hp >= 0 && hp < La.F_h, 7) ? (hp * C + src_row) * r + sv : 0;   // lifting: position
    float2 u0 = __ldg(Src + my_src);                   // the entry for u_w = 0 (all when sw = 1)
    if (my_conj) u0.y = -u0.y;
    my_a = make_float2((u0.x * my_pa.x - u0.y * my_pa.y) * scale, (u0.x * my_pa.y + u0.y * my_pa.x) * scale);
  }
  float2* out = dst + (size_t)(q0 - first) * C * n * m + row_off;
  const size_t vec_stride = (size_t)C * n * m;
  if (sw == 1 && (m & 1) == 0 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
    // 16-byte stores: a row is P = m/2 float4s; lane gl of a group of G lanes (the power of two
    // >= P, at most 32) writes float4s gl, gl + G, ... of one vector's row, and the warp's 32 / G
    // groups write the rows of as many consecutive vectors with one store instruction (two 32-entry
    // rows per instruction at m = 32). The column phase start and step are recomputed only when
    // the group's frequency changes.
    const int P = m >> 1;
    int G = 1;
    while (G < P && G < 32) G <<= 1;
    const int V = 32 / G, sub = lane / G, gl = lane - sub * G;
    unsigned lprev = 0xffffffffu, idx0 = 0, step = 0;
    for (int i0 = 0; i0 < nv; i0 += V) {
      const int iv = i0 + sub;
      const bool act = iv < nv;
      const int src_lane = iv & 31;
      const float2 a0 = make_float2(__shfl_sync(0xffffffffu, my_a.x, src_lane), __shfl_sync(0xffffffffu, my_a.y, src_lane));
      const unsigned l = __shfl_sync(0xffffffffu, my_l, src_lane);
      if (l != lprev) {
        lprev = l;
        idx0 = (l * (unsigned)(2 * gl)) % (unsigned)m;   // (l x2) mod m for x2 = 2 gl
        step = (l * (unsigned)(2 * G)) % (unsigned)m;
      }
      float4* o4 = reinterpret_cast<float4*>(out + (size_t)iv * vec_stride);
      unsigned idx = idx0;
      for (int q = gl; q < P; q += G) {
        unsigned i1 = idx + l;
        if (i1 >= (unsigned)m) i1 -= (unsigned)m;
        const float2 v0 = cmul(a0, La.tw_m[idx]), v1 = cmul(a0, La.tw_m[i1]);
        if (act) o4[q] = make_float4(v0.x, v0.y, v1.x, v1.y);
        idx += step;
        if (idx >= (unsigned)m) idx -= (unsigned)m;
      }
    }
    return;
  }
  // consecutive vectors mostly share the frequency: the column phase start and step are
  // recomputed only when l changes (l is warp-uniform, so is the branch)
  unsigned lprev = 0xffffffffu, idx0 = 0, step = 0;
  for (int i = 0; i < nv; ++i, out += vec_stride) {
    const float2 a0 = make_float2(__shfl_sync(0xffffffffu, my_a.x, i), __shfl_sync(0xffffffffu, my_a.y, i));
    const unsigned l = __shfl_sync(0xffffffffu, my_l, i);
    if (sw == 1) {
      if (l != lprev) {
        lprev = l;
        idx0 = (l * (unsigned)lane) % (unsigned)m;   // (l x2) mod m for x2 = lane
        step = (32u * l) % (unsigned)m;
      }
      unsigned idx = idx0;
      for (int z2 = lane; z2 < len; z2 += 32) {
        out[z2] = cmul(a0, La.tw_m[idx]);
        idx += step;
        if (idx >= (unsigned)m) idx -= (unsigned)m;
      }
    } else {
      const float2 pa = make_float2(__shfl_sync(0xffffffffu, my_pa.x, i), __shfl_sync(0xffffffffu, my_pa.y, i));
      const int conj = __shfl_sync(0xffffffffu, my_conj, i);
      const int64_t so = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)my_src, i);
      for (int z2 = lane; z2 < len; z2 += 32) {
        const int x2 = z2 / sw, uw = z2 - x2 * sw;
        float2 a = a0;
        if (uw != 0) {
          float2 u = __ldg(Src + so + (int64_t)uw * r);
          if (conj) u.y = -u.y;
          a = make_float2((u.x * pa.x - u.y * pa.y) * scale, (u.x * pa.y + u.y * pa.x) * scale);
        }
        out[z2] = cmul(a, La.tw_m[(l * (unsigned)x2) % (unsigned)m]);
      }
    }
  }
}

cudaError_t launch_expand(const LayerArgs& La, const float2* U, const float2* V, int64_t first,
                          int64_t count, float2* u_hat, float2* v_hat, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t groups = (count + kExpandVecs - 1) / kExpandVecs;
  if (groups > 65535) {
    // more vector groups than one grid dimension holds: split the range
    const int64_t per = (int64_t)65535 * kExpandVecs;
    for (int64_t q0 = 0; q0 < count; q0 += per) {
      const int64_t cnt = count - q0 < per ? count - q0 : per;
      cudaError_t e = launch_expand(La, U, V, first + q0, cnt,
                                    u_hat ? u_hat + (size_t)q0 * La.c_out * La.n * La.m : nullptr,
                                    v_hat ? v_hat + (size_t)q0 * La.c_in * La.n * La.m : nullptr, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const int64_t rows = (u_hat ? (int64_t)La.c_out * La.n : 0) + (v_hat ? (int64_t)La.c_w * La.sh * La.n : 0);
  if (rows <= 0) return cudaSuccess;
  if (rows > 0x7fffffffLL) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((rows + kExpandRowsPerCTA - 1) / kExpandRowsPerCTA), (unsigned)groups);
  expand_kernel<<<grid, 256, 0, s>>>(La, U, V, first, count, u_hat, v_hat);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- completion
// The X-side factor of a symbol (U for tall, V for wide; [M][N], column s = rank s) holds an
// exactly zero column where the forward found a negligible singular value (the cluster and
// rotation-log paths write them so). Its singular vector is any unit vector orthogonal to the
// other columns: start from the canonical vector e_k whose residual 1 - |row k|^2 (its squared
// distance from the span of the columns) is largest, which is at least (M - rank) / M, and
// orthogonalise it twice by classical Gram-Schmidt ("twice is enough"). Zero columns are
// completed in increasing order. One CTA per symbol; fixed-order sums (deterministic).
__global__ void __launch_bounds__(256) complete_kernel(float2* X, int M, int N) {
  __shared__ float res[512];
  __shared__ float2 v[512];
  __shared__ float2 cq[512];
  __shared__ unsigned char zero[512];
  __shared__ float rbest[8];
  __shared__ int kbest[8];
  __shared__ int nzero;
  float2* P = X + (size_t)blockIdx.x * M * N;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) nzero = 0;
  __syncthreads();
  // loops over rows keep four independent accumulators (four loads in flight per thread)
  for (int c = tid; c < N; c += blockDim.x) {
    float q[4] = {0.f, 0.f, 0.f, 0.f};
    int m = 0;
    for (; m + 4 <= M; m += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 x = P[(size_t)(m + u) * N + c];
        q[u] = fmaf(x.x, x.x, fmaf(x.y, x.y, q[u]));
      }
    }
    for (; m < M; ++m) {
      const float2 x = P[(size_t)m * N + c];
      q[0] = fmaf(x.x, x.x, fmaf(x.y, x.y, q[0]));
    }
    const float qq = (q[0] + q[1]) + (q[2] + q[3]);
    zero[c] = qq == 0.f;
    if (qq == 0.f) atomicAdd(&nzero, 1);
  }
  __syncthreads();
  if (nzero == 0) return;
  // squared distance of e_k from the span of the columns, one warp per row
  for (int k = wid; k < M; k += 8) {
    float q = 0.f;
    for (int c = lane; c < N; c += 32) {
      const float2 x = P[(size_t)k * N + c];
      q = fmaf(x.x, x.x, fmaf(x.y, x.y, q));
    }
    for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
    if (lane == 0) res[k] = 1.f - q;
  }
  __syncthreads();
  for (int d = 0; d < N; ++d) {
    if (!zero[d]) continue;                      // uniform: zero[] is shared
    // k* = argmax res (ties: smallest k)
    float rb = -1.f;
    int kb = 0;
    for (int k = tid; k < M; k += blockDim.x)
      if (res[k] > rb) { rb = res[k]; kb = k; }
    for (int off = 16; off > 0; off >>= 1) {
      const float orb = __shfl_xor_sync(0xffffffffu, rb, off);
      const int okb = __shfl_xor_sync(0xffffffffu, kb, off);
      if (orb > rb || (orb == rb && okb < kb)) { rb = orb; kb = okb; }
    }
    if (lane == 0) { rbest[wid] = rb; kbest[wid] = kb; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < 8; ++w)
        if (rbest[w] > rbest[0] || (rbest[w] == rbest[0] && kbest[w] < kbest[0])) {
          rbest[0] = rbest[w];
          kbest[0] = kbest[w];
        }
    }
    __syncthreads();
    const int ks = kbest[0];
    for (int m = tid; m < M; m += blockDim.x) v[m] = make_float2(m == ks ? 1.f : 0.f, 0.f);
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      // c = P^* v (one thread per column: coalesced rows), four row streams per thread
      for (int c = tid; c < N; c += blockDim.x) {
        float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
        int m = 0;
        for (; m + 4 <= M; m += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 x = P[(size_t)(m + u) * N + c], y = v[m + u];
            cr[u] = fmaf(x.x, y.x, fmaf(x.y, y.y, cr[u]));   // Re(conj(x) y)
            ci[u] = fmaf(x.x, y.y, fmaf(-x.y, y.x, ci[u]));  // Im(conj(x) y)
          }
        }
        for (; m < M; ++m) {
          const float2 x = P[(size_t)m * N + c], y = v[m];
          cr[0] = fmaf(x.x, y.x, fmaf(x.y, y.y, cr[0]));
          ci[0] = fmaf(x.x, y.y, fmaf(-x.y, y.x, ci[0]));
        }
        cq[c] = make_float2((cr[0] + cr[1]) + (cr[2] + cr[3]), (ci[0] + ci[1]) + (ci[2] + ci[3]));
      }
      __syncthreads();
      // v -= P c (one warp per row)
      for (int m = wid; m < M; m += 8) {
        float sr = 0.f, si = 0.f;
        for (int c = lane; c < N; c += 32) {
          const float2 x = P[(size_t)m * N + c], y = cq[c];
          sr = fmaf(x.x, y.x, fmaf(-x.y, y.y, sr));
          si = fmaf(x.x, y.y, fmaf(x.y, y.x, si));
        }
        for (int off = 16; off > 0; off >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, off);
          si += __shfl_xor_sync(0xffffffffu, si, off);
        }
        if (lane == 0) v[m] = make_float2(v[m].x - sr, v[m].y - si);
      }
      __syncthreads();
    }
    // normalise, write column d, update the residuals
    float q = 0.f;
    for (int m = tid; m < M; m += blockDim.x) q = fmaf(v[m].x, v[m].x, fmaf(v[m].y, v[m].y, q));
    for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
    if (lane == 0) rbest[wid] = q;
    __syncthreads();
    float nrm = 0.f;
    for (int w = 0; w < 8; ++w) nrm += rbest[w];
    const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
    for (int m = tid; m < M; m += blockDim.x) {
      const float2 u = make_float2(v[m].x * inv, v[m].y * inv);
      P[(size_t)m * N + d] = u;
      res[m] -= u.x * u.x + u.y * u.y;
    }
    __syncthreads();
  }
}

cudaError_t launch_complete(const LayerArgs& La, float2* X, int symbols, cudaStream_t s) {
  if (symbols <= 0) return cudaSuccess;
  if (La.M > 512 || La.N > 512) return cudaErrorInvalidValue;
  for (int h0 = 0; h0 < symbols; h0 += 65535) {
    const int cnt = symbols - h0 < 65535 ? symbols - h0 : 65535;
    complete_kernel<<<cnt, 256, 0, s>>>(X + (size_t)h0 * La.M * La.N, La.M, La.N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ----------------------------------------------------------------------------- backward
// Stage 1: G_h = U_h diag(g~_h) V_h^* (c_out x c_in complex) for every half-grid h, with
// g~ = g_f + g_fc for a conjugate pair, g_f for a self-conjugate f (full-grid dsigma), or the
// half-grid dsigma as is. Tiled batched complex GEMM over s: 32x32 output tile per CTA,
// 256 threads x 4 outputs, U/V chunks of 32 singular indices staged in shared memory.
__global__ void __launch_bounds__(256) backward_g_kernel(LayerArgs La, const float* dsigma,
                                                         int half_output, const float2* U,
                                                         const float2* V, int h_begin, float2* G) {
  __shared__ float2 Us[32][33];
  __shared__ float2 Vs[32][33];
  __shared__ float gs[32];
  const int h = h_begin + blockIdx.z;
  if (!LFA_DOK(La.dbg, h < La.F_h, 8)) return;           // backward G: symbol
  const int o0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
  const int r = La.r, co = La.c_out, ci = La.c_in;
  const int f = La.half[h];
  const int j = f / La.m, l = f - j * La.m;
  const int fc = ((La.n - j) % La.n) * La.m + (La.m - l) % La.m;
  const float* g_f = dsigma + (size_t)(half_output ? h : f) * r;
  const float* g_c = (!half_output && fc != f) ? dsigma + (size_t)fc * r : nullptr;
  const float2* Uh = U + (size_t)h * co * r;
  const float2* Vh = V + (size_t)h * ci * r;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  float2 acc[4] = {};
  for (int s0 = 0; s0 < r; s0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int rr = e >> 5, ss = e & 31;
      const int s = s0 + ss;
      Us[rr][ss] = (o0 + rr < co && s < r) ? Uh[(size_t)(o0 + rr) * r + s] : make_float2(0.f, 0.f);
      Vs[rr][ss] = (i0 + rr < ci && s < r) ? Vh[(size_t)(i0 + rr) * r + s] : make_float2(0.f, 0.f);
    }
    if (threadIdx.x < 32) {
      const int s = s0 + threadIdx.x;
      float g = 0.f;
      if (s < r) g = g_f[s] + (g_c ? g_c[s] : 0.f);
      gs[threadIdx.x] = g;
    }
    __syncthreads();
#pragma unroll 4
    for (int ss = 0; ss < 32; ++ss) {
      const float2 v = Vs[tx][ss];
      const float g = gs[ss];
      const float2 vg = make_float2(v.x * g, -v.y * g);  // g conj(v)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 u = Us[ty + 8 * k][ss];
        acc[k].x = fmaf(u.x, vg.x, fmaf(-u.y, vg.y, acc[k].x));
        acc[k].y = fmaf(u.x, vg.y, fmaf(u.y, vg.x, acc[k].y));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int o = o0 + ty + 8 * k, i = i0 + tx;
    if (o < co && i < ci) G[((size_t)blockIdx.z * co + o) * ci + i] = acc[k];
  }
}

// Stage 2: partial[c][o][i][a][b] = sum_{h in chunk c} Re(G_h[o,(i,u_ab)] exp(-2 pi i <k_h, q_ab>)),
// the phase split into its row factor (per thread) and column factor (per tap); at stride 1
// (i, u_ab) = i and q_ab = y_ab. One thread per (o, i, a) keeps the kw column taps in registers;
// the chunk's frequencies are summed in a fixed order (deterministic).
template <int KW>
__global__ void __launch_bounds__(128) backward_dw_kernel(LayerArgs La, const float2* G, int g_begin,
                                                          int chunk, int c_begin, float* partial) {
  const int CW = La.c_out * La.c_w;     // weight (o, i) pairs
  const int CC = La.c_out * La.c_in;    // symbol entries per G_h
  const int kh = La.kh, kw = La.kw;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = c_begin + blockIdx.y;
  if (tid >= CW * kh) return;
  const int e = tid / kh, a = tid - e * kh;
  const int o = e / La.c_w, ci = e - o * La.c_w;
  const int sh = La.sh, sw = La.sw;
  const int qa = floor_div(a - La.ph, sh), uh = (a - La.ph) - qa * sh;
  const int gcol = o * La.c_in + (ci * sh + uh) * sw;      // + u_w of the tap's column
  float acc[KW];
#pragma unroll
  for (int b = 0; b < KW; ++b) acc[b] = 0.f;
  const int h0 = c * chunk, h1 = min(La.F_h, h0 + chunk);
  for (int h = h0; h < h1; ++h) {
    const int f = La.half[h];
    const int j = f / La.m, l = f - j * La.m;
    const float2* Gh = G + (size_t)(h - g_begin) * CC + gcol;
    const float2 pa = La.tw_n[mod_pos(j * qa, La.n)];
    if (sw == 1) {
      const float2 g = Gh[0];
      const float2 ga = make_float2(g.x * pa.x + g.y * pa.y, g.y * pa.x - g.x * pa.y);   // G conj(pa)
#pragma unroll
      for (int b = 0; b < KW; ++b) {
        if (b < kw) {
          const float2 pb = La.tw_m[mod_pos(l * (b - La.pw), La.m)];
          acc[b] = fmaf(ga.x, pb.x, fmaf(ga.y, pb.y, acc[b]));   // Re(ga conj(pb))
        }
      }
    } else {
#pragma unroll
      for (int b = 0; b < KW; ++b) {
        if (b < kw) {
          const int qb = floor_div(b - La.pw, sw), uw = (b - La.pw) - qb * sw;
          const float2 g = Gh[uw];
          const float2 ga = make_float2(g.x * pa.x + g.y * pa.y, g.y * pa.x - g.x * pa.y);
          const float2 pb = La.tw_m[mod_pos(l * qb, La.m)];
          acc[b] = fmaf(ga.x, pb.x, fmaf(ga.y, pb.y, acc[b]));
        }
      }
    }
  }
  float* p = partial + ((size_t)c * CW + e) * (kh * kw) + (size_t)a * kw;
#pragma unroll
  for (int b = 0; b < KW; ++b)
    if (b < kw) p[b] = acc[b];
}

// Fused stages 1 + 2 for stride-1 layers with at most KK taps: one CTA per (chunk of frequencies,
// tile of 16 output x 64 input channels). Per frequency it forms its tile of G_h in registers
// (4 entries per thread: U rows scaled by g~ and V rows staged in shared memory, 32 singular
// indices at a time) and adds Re(G_h[o,i] conj(P_h[a,b])) for every tap to per-thread sums,
// with the k_h x k_w phases of the frequency in shared memory. Writes the same per-chunk partial
// sums as stage 2; no G round trip through memory. Fixed summation order (deterministic).
template <int KK>
__global__ void __launch_bounds__(256) backward_fused_kernel(LayerArgs La, const float* dsigma, int half_output,
                                                             const float2* U, const float2* V, int chunk,
                                                             float* partial) {
  constexpr int TO = 16, TI = 64;
  __shared__ float2 Us[TO][33];
  __shared__ float2 Vs[TI][33];
  __shared__ float2 sph[KK];
  const int r = La.r, co = La.c_out, ci = La.c_in, kk = La.kh * La.kw;
  const int o0 = blockIdx.y * TO, i0 = blockIdx.x * TI;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // entries (o0 + ty + 4 q, i0 + tx), q < 4
  const int c = blockIdx.z;
  const int h0 = c * chunk, h1 = min(La.F_h, h0 + chunk);
  const int nsc = (r + 31) / 32;                            // s-chunks per frequency
  const int iters = (h1 > h0 ? h1 - h0 : 0) * nsc;
  // staged tile of one (frequency, s-chunk): thread rows e = threadIdx.x + 256 k, s = e & 31
  float2 ur[2], vr[8];
  auto fetch = [&](int it) {
    const int h = h0 + it / nsc, s0 = (it % nsc) * 32;
    const int f = La.half[h];
    const int j = f / La.m, l = f - j * La.m;
    const int fc = ((La.n - j) % La.n) * La.m + (La.m - l) % La.m;
    const float* g_f = dsigma + (size_t)(half_output ? h : f) * r;
    const float* g_c = (!half_output && fc != f) ? dsigma + (size_t)fc * r : nullptr;
    const float2* Uh = U + (size_t)h * co * r;
    const float2* Vh = V + (size_t)h * ci * r;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = threadIdx.x + 256 * k, row = e >> 5, sg = s0 + (e & 31);
      float2 u = make_float2(0.f, 0.f);
      if (sg < r && o0 + row < co) {
        const float gs = g_f[sg] + (g_c ? g_c[sg] : 0.f);
        u = Uh[(size_t)(o0 + row) * r + sg];
        u = make_float2(u.x * gs, u.y * gs);
      }
      ur[k] = u;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int e = threadIdx.x + 256 * k, row = e >> 5, sg = s0 + (e & 31);
      vr[k] = (sg < r && i0 + row < ci) ? Vh[(size_t)(i0 + row) * r + sg] : make_float2(0.f, 0.f);
    }
  };
  float acc[4][KK];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int t = 0; t < KK; ++t) acc[q][t] = 0.f;
  float2 g[4];
  if (iters > 0) fetch(0);
  for (int it = 0; it < iters; ++it) {
    const int hh = h0 + it / nsc, sc = it % nsc;
    __syncthreads();                                       // the previous tile (and phases) are consumed
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = threadIdx.x + 256 * k;
      Us[e >> 5][e & 31] = ur[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int e = threadIdx.x + 256 * k;
      Vs[e >> 5][e & 31] = vr[k];
    }
    if (sc == 0) {
      const int f = La.half[hh];
      const int j = f / La.m, l = f - j * La.m;
      if (threadIdx.x < kk) sph[threadIdx.x] = tap_phase(La, j, l, threadIdx.x / La.kw, threadIdx.x % La.kw);
#pragma unroll
      for (int q = 0; q < 4; ++q) g[q] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (it + 1 < iters) fetch(it + 1);                     // the next tile's loads overlap this tile's math
#pragma unroll 8
    for (int ss = 0; ss < 32; ++ss) {
      const float2 v = Vs[tx][ss];
#pragma unroll
      for (int q = 0; q < 4; ++q) {                       // g += u conj(v)
        const float2 u = Us[ty + 4 * q][ss];
        g[q].x = fmaf(u.x, v.x, fmaf(u.y, v.y, g[q].x));
        g[q].y = fmaf(u.y, v.x, fmaf(-u.x, v.y, g[q].y));
      }
    }
    if (sc == nsc - 1) {
#pragma unroll
      for (int t = 0; t < KK; ++t) {
        if (t < kk) {
          const float2 p = sph[t];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q][t] = fmaf(g[q].x, p.x, fmaf(g[q].y, p.y, acc[q][t]));   // Re(g conj(p))
        }
      }
    }
  }
  const int CW = co * La.c_w;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int o = o0 + ty + 4 * q, i = i0 + tx;
    if (o >= co || i >= ci) continue;
    float* pp = partial + ((size_t)c * CW + (size_t)o * La.c_w + i) * kk;
#pragma unroll
    for (int t = 0; t < KK; ++t)
      if (t < kk) pp[t] = acc[q][t];
  }
}

// Whether the fused backward serves a layer, and its chunk count for a GPU of 152 SMs.
int fused_backward_chunks(const LayerArgs& La) {
  if (La.sh != 1 || La.sw != 1 || La.kh * La.kw > 25 || La.F_h <= 0) return 0;
  const int tiles = ((La.c_in + 63) / 64) * ((La.c_out + 15) / 16);
  int chunks = (4 * 152 + tiles - 1) / tiles;
  chunks = chunks < La.F_h ? chunks : La.F_h;
  chunks = chunks < 4096 ? chunks : 4096;
  return chunks < 1 ? 1 : chunks;
}

// Stage 3: dw = sum over chunks in order.
__global__ void __launch_bounds__(256) backward_reduce_kernel(const float* partial, int chunks,
                                                              int64_t total, float* dw) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += partial[(size_t)c * total + e];
  dw[e] = s;
}

cudaError_t launch_backward_reduce(const float* partial, int chunks, int64_t total, float* dw, cudaStream_t s) {
  backward_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(partial, chunks, total, dw);
  return cudaGetLastError();
}

// G holds g_cap symbols' G_h; the half grid is processed in blocks of whole chunks that fit.
cudaError_t launch_backward(const LayerArgs& La, const float* dsigma, int half_output,
                            const float2* U, const float2* V, float2* G, int64_t g_cap, float* partial,
                            int chunks, float* dw, cudaStream_t s, int* nkernels, unsigned int* queue,
                            Counters* ctr, int sms) {
  *nkernels = 0;
  const int CW = La.c_out * La.c_w;
  const int kk = La.kh * La.kw;
  // no frequencies (an empty shard of the half grid): the contribution is zero
  if (La.F_h <= 0) return cudaMemsetAsync(dw, 0, (size_t)CW * kk * sizeof(float), s);
  if (queue && ctr && G && g_cap >= 1 && sms > 0 && tc_backward_parts(La) > 0)
    return launch_backward_tc(La, dsigma, half_output, U, V, G, g_cap, partial, chunks, queue, ctr, dw, sms, s,
                              nkernels);
  if (La.sh == 1 && La.sw == 1 && kk <= 25 && chunks <= 65535) {
    // fused: G never leaves registers
    const int chunk = (La.F_h + chunks - 1) / chunks;
    const int nch = (La.F_h + chunk - 1) / chunk;
    dim3 grid((La.c_in + 63) / 64, (La.c_out + 15) / 16, nch);
    if (kk <= 1) backward_fused_kernel<1><<<grid, 256, 0, s>>>(La, dsigma, half_output, U, V, chunk, partial);
    else if (kk <= 9) backward_fused_kernel<9><<<grid, 256, 0, s>>>(La, dsigma, half_output, U, V, chunk, partial);
    else backward_fused_kernel<25><<<grid, 256, 0, s>>>(La, dsigma, half_output, U, V, chunk, partial);
    ++*nkernels;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)CW * kk;
    backward_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(partial, nch, total, dw);
    ++*nkernels;
    return cudaGetLastError();
  }
  const int chunk = (La.F_h + chunks - 1) / chunks;
  chunks = (La.F_h + chunk - 1) / chunk;
  int per_block = (int)(g_cap / chunk) < 1 ? 1 : (int)(g_cap / chunk);
  per_block = per_block * chunk > 65535 ? 65535 / chunk : per_block;   // gridDim.z limit
  if (per_block < 1) return cudaErrorInvalidValue;
  if ((int64_t)chunk > g_cap) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  for (int c0 = 0; c0 < chunks; c0 += per_block) {
    const int c1 = c0 + per_block < chunks ? c0 + per_block : chunks;
    const int h0 = c0 * chunk;
    const int h1 = c1 * chunk < La.F_h ? c1 * chunk : La.F_h;
    dim3 gg((La.c_in + 31) / 32, (La.c_out + 31) / 32, h1 - h0);
    backward_g_kernel<<<gg, 256, 0, s>>>(La, dsigma, half_output, U, V, h0, G);
    ++*nkernels;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 gd((CW * La.kh + 127) / 128, c1 - c0);
    if (La.kw <= 3) backward_dw_kernel<3><<<gd, 128, 0, s>>>(La, G, h0, chunk, c0, partial);
    else if (La.kw <= 7) backward_dw_kernel<7><<<gd, 128, 0, s>>>(La, G, h0, chunk, c0, partial);
    else backward_dw_kernel<15><<<gd, 128, 0, s>>>(La, G, h0, chunk, c0, partial);
    ++*nkernels;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t total = (int64_t)CW * La.kh * La.kw;
  backward_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(partial, chunks, total, dw);
  ++*nkernels;
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- regulariser
// loss = max(sigma) + lam * sum (sigma - 1)^2; dsigma = 2 lam (sigma - 1) + [first argmax].
// Pass 1: kRegBlocks CTAs write dsigma = 2 lam (sigma - 1) and one (max, first argmax, sum) per
// CTA over a contiguous slice; pass 2: one warp combines the partials in CTA order and adds the
// 1 at the argmax. Fixed-order reductions throughout (deterministic).
constexpr int kRegBlocks = 64;

__global__ void __launch_bounds__(256) regulariser_partial_kernel(const float* sigma, int64_t count, float lam,
                                                                  float* dsigma, float* pmax, long long* parg,
                                                                  float* psum) {
  __shared__ float smax[8];
  __shared__ long long sidx[8];
  __shared__ float ssum[8];
  const int64_t per = (count + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = (int64_t)blockIdx.x * per, e1 = e0 + per < count ? e0 + per : count;
  float best = -1.f;
  long long bi = 0x7fffffffffffffffll;
  float sum = 0.f;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const float v = sigma[e];
    if (v > best) { best = v; bi = e; }
    const float d = v - 1.f;
    sum = fmaf(d, d, sum);
    dsigma[e] = 2.f * lam * d;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    sum += __shfl_xor_sync(0xffffffffu, sum, off);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { smax[w] = best; sidx[w] = bi; ssum[w] = sum; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = -1.f, t = 0.f;
    long long ix = 0x7fffffffffffffffll;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      if (smax[i] > b || (smax[i] == b && sidx[i] < ix)) { b = smax[i]; ix = sidx[i]; }
      t += ssum[i];
    }
    pmax[blockIdx.x] = b;
    parg[blockIdx.x] = ix;
    psum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(32) regulariser_final_kernel(const float* pmax, const long long* parg,
                                                               const float* psum, int parts, int64_t count,
                                                               float lam, float* dsigma, float* loss) {
  // lane k combines parts k, k + 32, ... in order, then a fixed butterfly: deterministic
  const int lane = threadIdx.x;
  float b = -1.f, t = 0.f;
  long long ix = 0x7fffffffffffffffll;
  for (int i = lane; i < parts; i += 32) {
    if (pmax[i] > b || (pmax[i] == b && parg[i] < ix)) { b = pmax[i]; ix = parg[i]; }
    t += psum[i];
  }
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, b, off);
    const long long oi = __shfl_xor_sync(0xffffffffu, ix, off);
    if (ob > b || (ob == b && oi < ix)) { b = ob; ix = oi; }
    t += __shfl_xor_sync(0xffffffffu, t, off);
  }
  if (lane == 0) {
    if (ix >= 0 && ix < count) dsigma[ix] += 1.f;   // no index when every sigma is NaN
    if (loss) *loss = b + lam * t;
  }
}

cudaError_t launch_regulariser(const LayerArgs& La, int half_output, const float* sigma, float lam,
                               float* dsigma, float* loss, float* scratch, cudaStream_t s) {
  const int64_t count = (int64_t)(half_output ? La.F_h : La.n * La.m) * La.r;
  float* pmax = scratch;
  float* psum = scratch + kRegBlocks;
  long long* parg = reinterpret_cast<long long*>(scratch + 2 * kRegBlocks);
  regulariser_partial_kernel<<<kRegBlocks, 256, 0, s>>>(sigma, count, lam, dsigma, pmax, parg, psum);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  regulariser_final_kernel<<<1, 32, 0, s>>>(pmax, parg, psum, kRegBlocks, count, lam, dsigma, loss);
  return cudaGetLastError();
}

}  // namespace lfa

namespace lfa {

// ----------------------------------------------------------------------------- spectral editing
// g = mult(k) phi(sigma) / (n m): the upstream "gradient" whose backward is the projection of the
// edited operator onto the kernel taps. With the full-grid layout the backward folds k and -k;
// with the half-grid layout each row stands for mult(k) = 2 (conjugate pair) or 1 frequencies.
__global__ void __launch_bounds__(256) edit_values_kernel(LayerArgs La, int half_output, const float* sigma,
                                                           int mode, float a, float b, float* g) {
  const int rows = half_output ? La.F_h : La.n * La.m;
  const int r = La.r;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * r) return;
  const int row = (int)(e / r), s = (int)(e - (int64_t)row * r);
  const float v = sigma[e];
  float p;
  if (mode == 0) p = fminf(v, a);
  else if (mode == 1) p = fminf(fmaxf(v, a), b);
  else if (mode == 2) p = v >= a ? v : 0.f;
  else if (mode == 3) p = (float)s < rintf(a) ? v : 0.f;
  else p = v > a ? 1.f / v : 0.f;   // pseudo-inverse (correctly rounded reciprocal)
  float mult = 1.f;
  if (half_output) {
    const int f = La.half[row];
    const int j = f / La.m, l = f - j * La.m;
    const int fc = ((La.n - j) % La.n) * La.m + (La.m - l) % La.m;
    mult = fc != f ? 2.f : 1.f;
  }
  g[e] = mult * p / (float)(La.n * La.m);
}

cudaError_t launch_edit_values(const LayerArgs& La, int half_output, const float* sigma, int mode, float a,
                               float b, float* g, cudaStream_t s) {
  const int64_t total = (int64_t)(half_output ? La.F_h : La.n * La.m) * La.r;
  if (total <= 0) return cudaSuccess;
  edit_values_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(La, half_output, sigma, mode, a, b, g);
  return cudaGetLastError();
}

}  // namespace lfa
