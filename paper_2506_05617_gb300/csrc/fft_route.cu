// The FFT route to the symbols: the paper's comparison system (Sec. II and Sec. IV "Runtime
// Analysis", Table II), which obtains every symbol at once from a 2-D FFT of the kernel placed on
// the n x m grid, instead of assembling each symbol from its k_h x k_w taps (LFA).
//
// For each channel pair (o, i) the taps are placed at (a - p_h) mod n, (b - p_w) mod m (taps that
// alias are added), and cuFFT's batched real-to-complex forward transform gives
//   F_{oi}(j, l) = sum_x K_{oi}(x) exp(-2 pi i (j x1 / n + l x2 / m)) = conj(A_k[o][i]),
// for l <= m / 2. A half-grid frequency with l > m / 2 is read at (-j, -l), where
// A_k = conj(F(k)) = F(-k) (a real kernel). The symbols land in the layout of lfa_symbols
// ([F_h][c_out][c_in]) and the plain path's Jacobi kernels decompose them.
//
// The transform runs on cuFFT (a library); channel pairs are transformed in chunks whose
// workspace the plan allocates.
#include <cufft.h>

#include "half_grid.cuh"
#include "lfa_internal.cuh"

namespace lfa {

namespace {

__device__ __forceinline__ int mod_pos(int a, int n) {
  const int r = a % n;
  return r < 0 ? r + n : r;
}

// K[q][x1][x2] for the channel pairs q in [q0, q0 + count) (q = o c_in + i; stride-1 layers): the
// grid is zeroed, then every tap of w[o][i] is added at its offset mod (n, m) (aliasing taps add up).
__global__ void fft_zero_kernel(float* K, size_t total) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    K[e] = 0.f;
}

__global__ void fft_scatter_kernel(LayerArgs La, int q0, int count, float* K) {
  const int kk = La.kh * La.kw;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count * kk) return;
  const int ql = e / kk, t = e - ql * kk;
  const int a = t / La.kw, b = t - a * La.kw;
  const int x1 = mod_pos(a - La.ph, La.n), x2 = mod_pos(b - La.pw, La.m);
  atomicAdd(K + ((size_t)ql * La.n + x1) * La.m + x2, __ldg(La.w + (size_t)(q0 + ql) * kk + t));
}

// out[h][o][i] for the pairs of this chunk, from F [count][n][m/2 + 1].
__global__ void fft_gather_kernel(LayerArgs La, int q0, int count, const float2* F, float2* out) {
  const int mh = La.m / 2 + 1;
  const int CC = La.c_out * La.c_in;
  const size_t total = (size_t)La.F_h * count;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int ql = (int)(e % count);
    const int h = (int)(e / count);
    const int f = La.half[h];
    const int j = f / La.m, l = f - j * La.m;
    float2 v;
    if (l < mh) {
      v = F[((size_t)ql * La.n + j) * mh + l];
      v.y = -v.y;                                          // A_k = conj(F(k))
    } else {
      v = F[((size_t)ql * La.n + (La.n - j) % La.n) * mh + (La.m - l)];   // A_k = F(-k)
    }
    out[(size_t)h * CC + q0 + ql] = v;
  }
}

}  // namespace

// Pairs per chunk for a workspace of `bytes`: the real grid (4 n m) and the half spectrum
// (8 n (m/2 + 1)) of every pair.
int fft_chunk_pairs(const LayerArgs& La, size_t bytes) {
  const size_t per = (size_t)La.n * La.m * 4 + (size_t)La.n * (La.m / 2 + 1) * 8;
  const size_t c = bytes / per;
  const int CC = La.c_out * La.c_in;
  return (int)(c < (size_t)CC ? c : (size_t)CC);
}

cudaError_t fft_make_plan(const LayerArgs& La, int pairs, void** handle) {
  cufftHandle h;
  int dims[2] = {La.n, La.m};
  if (cufftPlanMany(&h, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, pairs) != CUFFT_SUCCESS)
    return cudaErrorUnknown;
  *handle = reinterpret_cast<void*>(static_cast<intptr_t>(h));
  return cudaSuccess;
}

void fft_destroy_plan(void* handle) {
  cufftDestroy(static_cast<cufftHandle>(reinterpret_cast<intptr_t>(handle)));
}

// All half-grid symbols of a stride-1 layer into out [F_h][c_out][c_in] through the FFT route.
// ws holds `pairs` channel pairs' real grids and spectra (fft_chunk_pairs); handle is a batched
// plan for `pairs` transforms (the last chunk runs a full batch over a partly stale tail, whose
// spectra are not gathered). Returns the number of kernels and transforms launched in *nk.
cudaError_t launch_fft_symbols(const LayerArgs& La, void* handle, int pairs, void* ws, float2* out, cudaStream_t s,
                               int* nk) {
  *nk = 0;
  const int CC = La.c_out * La.c_in;
  if (La.sh != 1 || La.sw != 1) return cudaErrorInvalidValue;
  cufftHandle h = static_cast<cufftHandle>(reinterpret_cast<intptr_t>(handle));
  if (cufftSetStream(h, s) != CUFFT_SUCCESS) return cudaErrorUnknown;
  float* K = static_cast<float*>(ws);
  float2* F = reinterpret_cast<float2*>(K + (size_t)pairs * La.n * La.m);
  const int kk = La.kh * La.kw;
  for (int q0 = 0; q0 < CC; q0 += pairs) {
    const int count = CC - q0 < pairs ? CC - q0 : pairs;
    const size_t total = (size_t)pairs * La.n * La.m;
    fft_zero_kernel<<<1216, 256, 0, s>>>(K, total);
    fft_scatter_kernel<<<(count * kk + 255) / 256, 256, 0, s>>>(La, q0, count, K);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (cufftExecR2C(h, K, reinterpret_cast<cufftComplex*>(F)) != CUFFT_SUCCESS) return cudaErrorUnknown;
    fft_gather_kernel<<<1216, 256, 0, s>>>(La, q0, count, F, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *nk += 3;
  }
  return cudaSuccess;
}

}  // namespace lfa
