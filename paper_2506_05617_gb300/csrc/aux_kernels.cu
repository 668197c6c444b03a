// Auxiliary kernels of the LFA SVD library (arXiv 2506.05617, Sec. III; strided layers as
// crystals):
//  * symbol assembly into memory (the plain path and lfa_symbols),
//  * lifting of symbol singular vectors to global singular vectors,
//  * the backward pass dL/dw,
//  * the spectral regulariser's dL/dsigma.
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

cudaError_t launch_symbols(const LayerArgs& La, float2* out, cudaStream_t s) {
  if (La.F_h <= 0) return cudaSuccess;
  symbols_kernel<<<La.F_h, 256, 0, s>>>(La, out);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- expansion
// u_hat[q][c][x1][x2] = U_f[c][s] exp(2 pi i (j x1/n + l x2/m)) / sqrt(nm), q = f*r + s
// (U^_k = F_k U_k, Sec. III). U_f = U[h] on the half grid, conj(U[h(fc)]) otherwise.
// For a stride, v_hat lives on the fine torus: v_hat[q][ci][sh x1 + uh][sw x2 + uw] takes
// row (ci, uh, uw) of V_f with the coarse mode of (x1, x2).
// Grid (element chunk, vector q); threads stride over the chunk's outputs (the last grid
// coordinate fastest: coalesced writes).
__device__ int half_index(const int32_t* half, int F_h, int f) {
  int lo = 0, hi = F_h - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (half[mid] < f) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256) expand_kernel(LayerArgs La, const float2* U, const float2* V,
                                                     int64_t first, float2* u_hat, float2* v_hat) {
  const int64_t q = first + blockIdx.y;
  const int r = La.r;
  const int f = (int)(q / r), s = (int)(q - (int64_t)f * r);
  const int j = f / La.m, l = f - j * La.m;
  const int fc = ((La.n - j) % La.n) * La.m + (La.m - l) % La.m;
  const bool conj = fc < f;
  const int h = half_index(La.half, La.F_h, conj ? fc : f);
  const int nm = La.n * La.m;
  const float scale = rsqrtf((float)nm);
  for (int pass = 0; pass < 2; ++pass) {
    const float2* Src = pass == 0 ? U : V;
    float2* dst = pass == 0 ? u_hat : v_hat;
    const int C = pass == 0 ? La.c_out : La.c_in;               // rows of the factor
    const int sh = pass == 0 ? 1 : La.sh, sw = pass == 0 ? 1 : La.sw;
    if (dst == nullptr || Src == nullptr) continue;
    const int G2 = La.m * sw;                                     // output grid sh n x sw m
    const int64_t G = (int64_t)La.n * sh * G2;
    const float2* col = Src + (size_t)h * C * r + s;
    float2* d = dst + (size_t)blockIdx.y * C * nm;
    const int64_t total = (int64_t)C * nm;                        // = (C / (sh sw)) * G
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t e0 = (int64_t)blockIdx.x * per, e1 = e0 + per < total ? e0 + per : total;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int c = (int)(e / G);
      const int64_t z = e - (int64_t)c * G;
      const int z1 = (int)(z / G2), z2 = (int)(z - (int64_t)z1 * G2);
      const int x1 = z1 / sh, uh = z1 - x1 * sh, x2 = z2 / sw, uw = z2 - x2 * sw;
      float2 u = __ldg(col + (size_t)((c * sh + uh) * sw + uw) * r);
      if (conj) u.y = -u.y;
      const float2 ph = cmul(La.tw_n[(int)(((int64_t)j * x1) % La.n)],
                             La.tw_m[(int)(((int64_t)l * x2) % La.m)]);
      const float2 v = cmul(u, ph);
      d[e] = make_float2(v.x * scale, v.y * scale);
    }
  }
}

cudaError_t launch_expand(const LayerArgs& La, const float2* U, const float2* V, int64_t first,
                          int64_t count, float2* u_hat, float2* v_hat, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (count > 65535) {
    // more vectors than one grid dimension holds: split the range
    for (int64_t q0 = 0; q0 < count; q0 += 65535) {
      const int64_t cnt = count - q0 < 65535 ? count - q0 : 65535;
      cudaError_t e = launch_expand(La, U, V, first + q0, cnt,
                                    u_hat ? u_hat + (size_t)q0 * La.c_out * La.n * La.m : nullptr,
                                    v_hat ? v_hat + (size_t)q0 * La.c_in * La.n * La.m : nullptr, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const int64_t per_vec = (int64_t)(La.c_out > La.c_in ? La.c_out : La.c_in) * La.n * La.m;
  int64_t chunks = (per_vec + 8191) / 8192;                 // ~32 elements per thread
  const int64_t want = 4 * 152 * 4;                          // enough CTAs to fill the GPU
  if (chunks * count > want) chunks = (want + count - 1) / count;
  if (chunks < 1) chunks = 1;
  dim3 grid((unsigned)chunks, (unsigned)count);
  expand_kernel<<<grid, 256, 0, s>>>(La, U, V, first, u_hat, v_hat);
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
  for (int c = tid; c < N; c += blockDim.x) {
    float q = 0.f;
    for (int m = 0; m < M; ++m) {
      const float2 x = P[(size_t)m * N + c];
      q = fmaf(x.x, x.x, fmaf(x.y, x.y, q));
    }
    zero[c] = q == 0.f;
    if (q == 0.f) atomicAdd(&nzero, 1);
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
      // c = P^* v (one thread per column: coalesced rows)
      for (int c = tid; c < N; c += blockDim.x) {
        float cr = 0.f, ci = 0.f;
        for (int m = 0; m < M; ++m) {
          const float2 x = P[(size_t)m * N + c], y = v[m];
          cr = fmaf(x.x, y.x, fmaf(x.y, y.y, cr));       // Re(conj(x) y)
          ci = fmaf(x.x, y.y, fmaf(-x.y, y.x, ci));      // Im(conj(x) y)
        }
        cq[c] = make_float2(cr, ci);
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

// Stage 3: dw = sum over chunks in order.
__global__ void __launch_bounds__(256) backward_reduce_kernel(const float* partial, int chunks,
                                                              int64_t total, float* dw) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += partial[(size_t)c * total + e];
  dw[e] = s;
}

// G holds g_cap symbols' G_h; the half grid is processed in blocks of whole chunks that fit.
cudaError_t launch_backward(const LayerArgs& La, const float* dsigma, int half_output,
                            const float2* U, const float2* V, float2* G, int64_t g_cap, float* partial,
                            int chunks, float* dw, cudaStream_t s, int* nkernels) {
  *nkernels = 0;
  if (La.F_h <= 0) return cudaSuccess;
  const int CW = La.c_out * La.c_w;
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
// One CTA of 1024 threads per layer; fixed-order tree reductions (deterministic).
__global__ void __launch_bounds__(1024) regulariser_kernel(const float* sigma, int64_t count, float lam,
                                                           float* dsigma, float* loss) {
  __shared__ float smax[32];
  __shared__ long long sidx[32];
  __shared__ float ssum[32];
  float best = -1.f;
  long long bi = 0x7fffffffffffffffll;
  float sum = 0.f;
  for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
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
    float b = -1.f, s = 0.f;
    long long ix = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      if (smax[i] > b || (smax[i] == b && sidx[i] < ix)) { b = smax[i]; ix = sidx[i]; }
      s += ssum[i];
    }
    if (count > 0) dsigma[ix] += 1.f;
    if (loss) *loss = b + lam * s;
  }
}

cudaError_t launch_regulariser(const LayerArgs& La, int half_output, const float* sigma, float lam,
                               float* dsigma, float* loss, cudaStream_t s) {
  const int64_t count = (int64_t)(half_output ? La.F_h : La.n * La.m) * La.r;
  regulariser_kernel<<<1, 1024, 0, s>>>(sigma, count, lam, dsigma, loss);
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
  else p = (float)s < rintf(a) ? v : 0.f;
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
