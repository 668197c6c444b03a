// lfa_svd_backward_noalloc: the backward pass (dL/dw from dL/dsigma) for callers that
// cannot allocate device memory. It needs no plan (creating a plan allocates) and
// takes its scratch space -- the twiddle tables, the per-frequency G_k block workspace
// and the per-chunk partial sums -- from one fixed array in the library's own
// device image instead of cudaMalloc.
//
// Who cannot allocate: a caller whose device memory is wholly owned by another
// allocator (a framework's caching allocator, or a serving runtime that reserves
// HBM at start-up and hands out fixed budgets) gets no room for a private
// cudaMalloc; and a caller in a latency-critical loop cannot pay for
// cudaMalloc/cudaFree, which may synchronise the device.
//
// The scratch array is LFA_NOALLOC_SCRATCH_BYTES large. Every GPU that loads this
// library holds it until the process exits. All calls share it and it keeps the last
// call's contents; nothing in it has to start at zero (each call writes every byte it
// later reads). Calls that overlap on the GPU (on different streams, or from different
// host threads without ordering) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/lfa.h"
#include "lfa_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)LFA_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch itself. In host code this name is only a host-side stand-in for the
// device array, never a device address: the kernels get the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
struct ScratchAddr {
  unsigned long long ctx_id;   // driver context the address belongs to (0: unknown)
  void* ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

// The unique id of the calling thread's current driver context, or 0 when it cannot be read.
// The driver calls are reached through the runtime's entry-point query, so the library does not
// link the driver library itself.
unsigned long long current_context_id() {
  typedef int (*GetCurrentFn)(void**);
  typedef int (*GetIdFn)(void*, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(f);
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == 0 && ctx != nullptr && get_id(ctx, &id) == 0) return id;
  return 0;
}

// Set-up, once per device and driver context, with that device current: the device address of
// the array. A device reset (or another context made current) gives a new context id, and the
// address is looked up again.
cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  const unsigned long long id = current_context_id();
  ScratchAddr& a = g_scratch[dev];
  if (a.ptr == nullptr || id == 0 || id != a.ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    a.ptr = p;
    a.ctx_id = current_context_id();   // the lookup above makes the primary context current if none was
  }
  *out = static_cast<unsigned char*>(a.ptr);
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// T[t] = exp(2 pi i t / n), evaluated in fp64 on the device and rounded to fp32.
__global__ void twiddle_kernel(float2* tw_n, int n, float2* tw_m, int m) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    double s, c;
    sincospi(2.0 * (double)t / (double)n, &s, &c);
    tw_n[t] = make_float2((float)c, (float)s);
  }
  if (t < m) {
    double s, c;
    sincospi(2.0 * (double)t / (double)m, &s, &c);
    tw_m[t] = make_float2((float)c, (float)s);
  }
}

// The half grid in increasing row-major order, written arithmetically: row 0 and
// (n even) row n/2 hold l = 0 .. floor(m/2); rows 1 .. ceil(n/2)-1 hold all l.
__global__ void half_grid_kernel(int32_t* half, int n, int m, int F_h) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= F_h) return;
  const int c0 = m / 2 + 1;
  const int full_rows = (n - 1) / 2;       // rows j with 0 < j < n - j
  int f;
  if (h < c0) {
    f = h;
  } else if (h < c0 + full_rows * m) {
    const int q = h - c0;
    f = (1 + q / m) * m + q % m;
  } else {
    f = (n / 2) * m + (h - c0 - full_rows * m);
  }
  half[h] = f;
}

}  // namespace

extern "C" lfa_status_t lfa_svd_backward_noalloc(const lfa_layer_desc_t* layer, uint32_t flags,
                                                 const float* dsigma, const float* U, const float* V,
                                                 float* dw, void* stream) {
  using namespace lfa;
  if (layer == nullptr || dsigma == nullptr || U == nullptr || V == nullptr || dw == nullptr)
    return LFA_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)LFA_HALF_OUTPUT) return LFA_ERR_INVALID_ARG;
  const lfa_layer_desc_t& d = *layer;
  LayerArgs La;
  if (!set_geometry(La, d.c_out, d.c_in, d.kh, d.kw, d.n, d.m, d.pad_h, d.pad_w, d.stride_h, d.stride_w))
    return LFA_ERR_INVALID_ARG;
  La.w = nullptr;
  La.sigma = nullptr;
  La.U = nullptr;
  La.V = nullptr;
  La.symbols = nullptr;
  La.dbg = nullptr;
  const int s_self = (1 + (d.n % 2 == 0)) * (1 + (d.m % 2 == 0));
  La.F_h = (int)(((int64_t)d.n * d.m + s_self) / 2);
  La.item_begin = 0;
  La.tol2 = 0.f;

  // scratch layout: half-grid list | twiddles n | twiddles m | partial sums | G workspace.
  const int64_t CW = (int64_t)La.c_out * La.c_w;    // weight (o, i) pairs
  const int64_t CC = (int64_t)La.c_out * La.c_in;   // symbol entries (>= weight pairs)
  const int64_t kk = (int64_t)d.kh * d.kw;
  const size_t slab = (size_t)(CW * kk * 4);        // partial sums of one chunk
  const size_t fixed = align256((size_t)La.F_h * 4) + align256((size_t)d.n * 8) + align256((size_t)d.m * 8);
  if (fixed >= kScratchBytes / 2) return LFA_ERR_UNSUPPORTED;
  int64_t chunks = 0, chunk = 0, g_cap = 0;
  size_t part_bytes = 0;
  const int fused = fused_backward_chunks(La);
  if (fused > 0) {
    // Stride-1 layers with at most 25 taps take the fused route: G_k never leaves registers, so
    // the whole array after the tables holds partial sums. The chunk count is the planned
    // backward's (same rounding order) when its partials fit, else the largest count that fits.
    const int64_t fit = (int64_t)((kScratchBytes - fixed) / slab);
    if (fit < 1) return LFA_ERR_UNSUPPORTED;                      // one partial slab does not fit
    chunks = fused < fit ? fused : fit;
    chunk = (La.F_h + chunks - 1) / chunks;
    chunks = (La.F_h + chunk - 1) / chunk;
    part_bytes = align256((size_t)chunks * slab);
  } else {
    // G route: the partial sums get at most half the array; G gets the rest and must hold one
    // chunk of G_k blocks. The planned backward's chunk count is used when it fits.
    const size_t part_budget = kScratchBytes / 2 - fixed;
    const int64_t fit = (int64_t)(part_budget / slab);
    if (fit < 1) return LFA_ERR_UNSUPPORTED;                      // one partial slab does not fit
    int64_t want = (155648 + CC - 1) / CC;                          // the plan's count for a roomy G
    want = want < La.F_h ? want : La.F_h;
    want = want < 4096 ? want : 4096;
    chunks = want < fit ? want : fit;
    chunk = (La.F_h + chunks - 1) / chunks;
    if (chunk > 65535) return LFA_ERR_UNSUPPORTED;
    chunks = (La.F_h + chunk - 1) / chunk;
    part_bytes = align256((size_t)chunks * slab);
    const size_t g_bytes = kScratchBytes - fixed - part_bytes;
    g_cap = (int64_t)(g_bytes / (size_t)(CC * 8));
    if (g_cap < chunk) {
      // more, smaller chunks leave more room for G: take the count that balances the two
      for (int64_t c = chunks + 1; c <= fit && c <= La.F_h; ++c) {
        const int64_t ch = (La.F_h + c - 1) / c;
        const size_t pb = align256((size_t)((La.F_h + ch - 1) / ch) * slab);
        if (pb > part_budget) break;
        if ((int64_t)((kScratchBytes - fixed - pb) / (size_t)(CC * 8)) >= ch) {
          chunk = ch;
          chunks = (La.F_h + ch - 1) / ch;
          part_bytes = pb;
          break;
        }
      }
      g_cap = (int64_t)((kScratchBytes - fixed - part_bytes) / (size_t)(CC * 8));
      if (g_cap < chunk) return LFA_ERR_UNSUPPORTED;                // one chunk of G does not fit
    }
  }

  unsigned char* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LFA_ERR_OOM : LFA_ERR_CUDA;
  int32_t* half = reinterpret_cast<int32_t*>(base);
  float2* tw_n = reinterpret_cast<float2*>(base + align256((size_t)La.F_h * 4));
  float2* tw_m = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(tw_n) + align256((size_t)d.n * 8));
  float* partial = reinterpret_cast<float*>(base + fixed);
  float2* G = g_cap > 0 ? reinterpret_cast<float2*>(base + fixed + part_bytes) : nullptr;
  La.half = half;
  La.tw_n = tw_n;
  La.tw_m = tw_m;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nm_max = d.n > d.m ? d.n : d.m;
  // cudaLaunchKernel returns the status of this launch alone (cudaGetLastError would also report,
  // and clear, an error left behind by unrelated earlier work)
  {
    int n_ = d.n, m_ = d.m;
    void* args[] = {&tw_n, &n_, &tw_m, &m_};
    e = cudaLaunchKernel(reinterpret_cast<const void*>(twiddle_kernel), dim3((nm_max + 255) / 256), dim3(256), args,
                         0, s);
  }
  if (e == cudaSuccess) {
    int n_ = d.n, m_ = d.m, fh = La.F_h;
    void* args[] = {&half, &n_, &m_, &fh};
    e = cudaLaunchKernel(reinterpret_cast<const void*>(half_grid_kernel), dim3((La.F_h + 255) / 256), dim3(256),
                         args, 0, s);
  }
  if (e == cudaSuccess) {
    int nk = 0;
    e = launch_backward(La, dsigma, (flags & LFA_HALF_OUTPUT) ? 1 : 0, reinterpret_cast<const float2*>(U),
                        reinterpret_cast<const float2*>(V), G, g_cap, partial, (int)chunks, dw, s, &nk);
  }
  return e == cudaSuccess ? LFA_OK : LFA_ERR_CUDA;
}
