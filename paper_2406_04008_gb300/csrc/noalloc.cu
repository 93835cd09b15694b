// collage_uniform_term_noalloc: the even-distribution term and its adjoint for one image, with all
// scratch in a file-scope device array instead of memory from cudaMalloc.
//
// Who needs it: callers whose device memory belongs to someone else -- a framework's caching
// allocator or a fixed arena they must not bypass -- and real-time loops that may not pay for
// cudaMalloc / cudaFree (both can synchronise the device).  They pass in the rendered image, the
// container coverage and the two outputs; everything else lives in g_noalloc_scratch, which every
// GPU that loads libcollage holds until the process exits.
#include <mutex>
#include <string>

#include "collage.h"
#include "internal.h"

namespace collage {

constexpr int kNoAllocMaxDT = (1024 / 32) * (1024 / 32);  // 32 x 32 dilation tiles
// layout: [the adjoint's staged words: uint32 x max pixels][tile partials: float x max tiles]
//         [small ints: status, res, dilation-tile base (2), pixel base as long long (2)]
constexpr size_t kOffLossU = sizeof(uint32_t) * COLLAGE_NOALLOC_MAX_PIXELS;
constexpr size_t kOffInts = kOffLossU + sizeof(float) * kNoAllocMaxDT;
constexpr size_t kNoAllocBytes = kOffInts + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocInts {
  int status;
  int res;
  int dtile_base[2];
  long long pix_base[2];
};

// Per call: the single-problem level arrays and a cleared status word.
__global__ void k_noalloc_setup(int res) {
  NoAllocInts* s = reinterpret_cast<NoAllocInts*>(g_noalloc_scratch + kOffInts);
  const int nd = (res + 31) / 32;
  s->status = 0;
  s->res = res;
  s->dtile_base[0] = 0;
  s->dtile_base[1] = nd * nd;
  s->pix_base[0] = 0;
  s->pix_base[1] = (long long)res * res;
}

// Fixed-order sum of the per-tile partials into the caller's loss.
__global__ void k_noalloc_sum(int n_tiles, float* out) {
  const float* part = reinterpret_cast<const float*>(g_noalloc_scratch + kOffLossU);
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n_tiles; i += blockDim.x) s += part[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
    out[0] = (float)t;
  }
}

}  // namespace collage

using namespace collage;

namespace {
std::mutex g_mu;
unsigned char* g_scratch_ptr[128] = {nullptr};  // per device ordinal
}  // namespace

extern "C" collage_status collage_uniform_term_noalloc(void* stream, int res, int n_dilations,
                                                       const float* h_dil_weight,
                                                       const float* d_ihat, const float* d_cov,
                                                       float* d_loss, float* d_grad_occ) {
  if (res < 1 || (long long)res * res > COLLAGE_NOALLOC_MAX_PIXELS) return COLLAGE_ERR_INVALID_ARG;
  if (n_dilations < 1 || n_dilations > kMaxDil || !h_dil_weight || !d_ihat || !d_cov || !d_loss ||
      !d_grad_occ)
    return COLLAGE_ERR_INVALID_ARG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) return COLLAGE_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    // once per device, with that device current: the device address of the scratch array, and
    // the dynamic shared-memory limit of every dilation kernel (a per-device function attribute;
    // each kernel's limit is a constant of its kernel count, so no later call changes it)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return COLLAGE_ERR_CUDA;
      if (prepare_dilate(kMaxDil) != cudaSuccess) return COLLAGE_ERR_CUDA;
      g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_scratch_ptr[dev];
  }
  NoAllocInts* ints = reinterpret_cast<NoAllocInts*>(base + kOffInts);
  const int nd = (res + 31) / 32;
  Dev d{};
  d.n_probs = 1;
  d.prob_res = &ints->res;
  d.prob_dtile_base = ints->dtile_base;
  d.prob_pix_base = ints->pix_base;
  d.total_dtiles = nd * nd;
  d.total_pix = (long long)res * res;
  d.status = &ints->status;
  d.img_I = const_cast<float*>(d_ihat);
  d.covc = const_cast<float*>(d_cov);
  d.gOu = d_grad_occ;
  d.dil_g = reinterpret_cast<uint32_t*>(base);
  d.lossU = reinterpret_cast<float*>(base + kOffLossU);
  d.L.n_dil = n_dilations;
  d.L.gamma = 1.0f;
  for (int k = 0; k < kMaxDil; ++k) d.L.dil_w[k] = k < n_dilations ? h_dil_weight[k] : 0.0f;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_noalloc_setup<<<1, 1, 0, s>>>(res);
  if ((e = cudaGetLastError()) == cudaSuccess) e = launch_dilate(d, s, false);
  if (e == cudaSuccess) e = launch_dilate(d, s, true);
  if (e == cudaSuccess) {
    k_noalloc_sum<<<1, 1024, 0, s>>>(nd * nd, d_loss);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? COLLAGE_OK : COLLAGE_ERR_CUDA;
}
