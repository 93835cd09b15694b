// Transform (Eq. 2) and tile binning: per-element tile rectangles, an exclusive scan of the pair
// counts, key emission, a stable LSD radix sort of (tile key, emit position) pairs, and per-tile
// [begin, end) ranges.  Integer work is bit-exact: the tile rectangle follows a fixed float
// formula (see bin_rect), emission is element-major, and the sort is stable, so each tile lists
// its elements in increasing element order.
#include <cfloat>

#include "internal.h"

namespace collage {

__device__ __forceinline__ float warp_min(float x) {
  for (int o = 16; o; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ float warp_max(float x) {
  for (int o = 16; o; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Tile rectangle of one element, float arithmetic in a fixed order with explicit round-to-nearest
// intrinsics (no contraction):
//   R_px = (s * r_bin) * res, c = t * res, m = ((rho + pad) + hw * res) + 1,
//   [floor(((c - R_px) - m) / T), floor(((c + R_px) + m) / T)] clipped to the grid's tiles.
// The circle of radius s * r_bin about t holds the whole outline because r_bin bounds every
// control point and a Bezier curve stays inside the convex hull of its control points.
__device__ int4 bin_rect(float4 q, float rbin, float hw, int res, int T, float rho, float pad) {
  const float fres = (float)res;
  const float Rpx = __fmul_rn(__fmul_rn(q.w, rbin), fres);
  const float cx = __fmul_rn(q.x, fres), cy = __fmul_rn(q.y, fres);
  const float m = __fadd_rn(__fadd_rn(__fadd_rn(rho, pad), __fmul_rn(hw, fres)), 1.0f);
  const float x0 = __fsub_rn(__fsub_rn(cx, Rpx), m), x1 = __fadd_rn(__fadd_rn(cx, Rpx), m);
  const float y0 = __fsub_rn(__fsub_rn(cy, Rpx), m), y1 = __fadd_rn(__fadd_rn(cy, Rpx), m);
  const float fT = (float)T;
  const float fx0 = floorf(__fdiv_rn(x0, fT)), fx1 = floorf(__fdiv_rn(x1, fT));
  const float fy0 = floorf(__fdiv_rn(y0, fT)), fy1 = floorf(__fdiv_rn(y1, fT));
  const int nt = (res + T - 1) / T;
  const float lim = (float)(nt - 1);
  int4 r = make_int4(0, 0, -1, -1);
  if (!(fx1 >= 0.0f && fy1 >= 0.0f && fx0 <= lim && fy0 <= lim)) return r;  // also NaN
  r.x = fx0 < 0.0f ? 0 : (int)fx0;
  r.y = fy0 < 0.0f ? 0 : (int)fy0;
  r.z = fx1 > lim ? nt - 1 : (int)fx1;
  r.w = fy1 > lim ? nt - 1 : (int)fy1;
  return r;
}

// One warp per element: vertices relative to the translation, in pixels, computed in double and
// rounded once (Eq. 2 without the translation); translation in pixels as a float hi/lo pair; pixel
// bounding box grown by the coverage margin; tile rectangle and pair count.
__global__ void k_transform(Dev d, int zero_grad) {
  const int g = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= d.n_elems) return;
  const int p = d.elem_prob[g];
  const int res = d.prob_res[p];
  const float4 q = d.q[g];
  double sn, c;
  sincos((double)q.z, &sn, &c);
  const double sc = (double)q.w * (double)res;
  const int v0 = d.elem_voff[g], v1 = d.elem_voff[g + 1];
  float xmin = FLT_MAX, ymin = FLT_MAX, xmax = -FLT_MAX, ymax = -FLT_MAX;
  for (int k = v0 + lane; k < v1; k += 32) {
    const float2 v = d.vloc[k];
    const double x = sc * (c * (double)v.x - sn * (double)v.y);
    const double y = sc * (sn * (double)v.x + c * (double)v.y);
    const float2 r = make_float2((float)x, (float)y);
    d.vrel[k] = r;
    xmin = fminf(xmin, r.x);
    xmax = fmaxf(xmax, r.x);
    ymin = fminf(ymin, r.y);
    ymax = fmaxf(ymax, r.y);
  }
  xmin = warp_min(xmin);
  ymin = warp_min(ymin);
  xmax = warp_max(xmax);
  ymax = warp_max(ymax);
  if (lane != 0) return;
  const double tx = (double)q.x * res, ty = (double)q.y * res;
  const float hx = (float)tx, hy = (float)ty;
  d.tpx[g] = make_float4(hx, hy, (float)(tx - (double)hx), (float)(ty - (double)hy));
  const bool closed = d.elem_closed[g] != 0;
  const float hw = closed ? 0.0f : d.elem_hw[g];
  const float m = d.L.rho_px + d.L.pad_px + hw * (float)res + 0.01f;
  d.bbox[g] = make_float4(hx + xmin - m, hy + ymin - m, hx + xmax + m, hy + ymax + m);
  const bool finite = isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w) && q.w > 0.0f;
  int4 r = make_int4(0, 0, -1, -1);
  if (finite) r = bin_rect(q, d.elem_rbin[g], hw, res, d.tile, d.L.rho_px, d.L.pad_px);
  else atomicOr(d.status, kStatusBadParam);
  d.rect[g] = r;
  d.cnt[g] = (r.z >= r.x && r.w >= r.y) ? (r.z - r.x + 1) * (r.w - r.y + 1) : 0;
  if (zero_grad) d.dq[g] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Exclusive scan of the pair counts, one block of 1024 threads (contiguous chunk per thread).
__global__ void __launch_bounds__(1024) k_scan(Dev d) {
  __shared__ int wsum[32];
  const int n = d.n_elems, t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = min(t * per, n), e = min(b + per, n);
  int s = 0;
  for (int i = b; i < e; ++i) s += d.cnt[i];
  // block exclusive scan of s
  const int lane = t & 31, w = t >> 5;
  int x = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int ws = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += y;
    }
    wsum[lane] = ws;  // inclusive
  }
  __syncthreads();
  int run = x - s + (w > 0 ? wsum[w - 1] : 0);
  for (int i = b; i < e; ++i) {
    d.off[i] = run;
    run += d.cnt[i];
  }
  if (t == 1023) {
    d.off[n] = run;
    *d.total_pairs = run;
    if (run > d.cap) atomicOr(d.status, kStatusOverflow);
  }
}

// Keys: global tile id (problem tile base + row-major tile index); values: emit position.
__global__ void k_emit(Dev d) {
  const int g = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= d.n_elems || (*d.status & kStatusOverflow)) return;
  const int c = d.cnt[g];
  if (c == 0) return;
  const int4 r = d.rect[g];
  const int w = r.z - r.x + 1;
  const int base = d.off[g], p = d.elem_prob[g];
  const int tb = d.prob_tile_base[p], ntx = d.prob_ntx[p];
  for (int i = lane; i < c; i += 32) {
    const int ty = r.y + i / w, tx = r.x + i % w;
    d.keys0[base + i] = (uint32_t)(tb + ty * ntx + tx);
    d.vals0[base + i] = (uint32_t)(base + i);
    d.elem_of[base + i] = g;
  }
}

__device__ __forceinline__ int sort_count(const Dev& d) {
  if (*d.status & kStatusOverflow) return 0;
  return *d.total_pairs;
}

// Radix pass, step 1: per-block digit histogram of a contiguous chunk.
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(Dev d, int shift, const uint32_t* keys) {
  __shared__ int h[kSortBins];
  const int n = sort_count(d), G = gridDim.x, b = blockIdx.x;
  for (int i = threadIdx.x; i < kSortBins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int chunk = (n + G - 1) / G;
  const int s = min(b * chunk, n), e = min(s + chunk, n);
  for (int i = s + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&h[(keys[i] >> shift) & (kSortBins - 1)], 1);
  __syncthreads();
  for (int i = threadIdx.x; i < kSortBins; i += blockDim.x) d.sort_hist[i * G + b] = (uint32_t)h[i];
}

// Radix pass, step 2: exclusive scan of the digit-major histogram (one block).
__global__ void __launch_bounds__(1024) k_sort_scan(Dev d, int G) {
  __shared__ uint32_t wsum[32];
  const int n = kSortBins * G, t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = min(t * per, n), e = min(b + per, n);
  uint32_t s = 0;
  for (int i = b; i < e; ++i) s += d.sort_hist[i];
  const int lane = t & 31, w = t >> 5;
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t ws = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += y;
    }
    wsum[lane] = ws;
  }
  __syncthreads();
  uint32_t run = x - s + (w > 0 ? wsum[w - 1] : 0u);
  for (int i = b; i < e; ++i) {
    const uint32_t c = d.sort_hist[i];
    d.sort_hist[i] = run;
    run += c;
  }
}

// Radix pass, step 3: stable scatter.  A block walks its chunk in rounds of 256 keys in input
// order; ranks among equal digits come from warp match masks (lower lanes first) and a per-digit
// prefix over the block's warps, so equal keys keep their input order.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(Dev d, int shift, const uint32_t* kin,
                                                               const uint32_t* vin, uint32_t* kout,
                                                               uint32_t* vout) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t run[kSortBins];
  __shared__ uint32_t wcnt[W][kSortBins];
  const int n = sort_count(d), G = gridDim.x, b = blockIdx.x;
  const int chunk = (n + G - 1) / G;
  const int s = min(b * chunk, n), e = min(s + chunk, n);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int i = t; i < kSortBins; i += blockDim.x) run[i] = d.sort_hist[i * G + b];
  for (int base = s; base < e; base += kSortThreads) {
    for (int i = t; i < W * kSortBins; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int i = base + t;
    const bool live = i < e;
    uint32_t key = 0, val = 0, dig = 0xffffffffu;
    if (live) {
      key = kin[i];
      val = vin[i];
      dig = (key >> shift) & (kSortBins - 1);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (live && rank == 0) wcnt[w][dig] = (uint32_t)__popc(peers);
    __syncthreads();
    for (int g = t; g < kSortBins; g += blockDim.x) {  // prefix over warps, per digit
      uint32_t r = run[g];
      for (int ww = 0; ww < W; ++ww) {
        const uint32_t c = wcnt[ww][g];
        wcnt[ww][g] = r;
        r += c;
      }
      run[g] = r;
    }
    __syncthreads();
    if (live) {
      const uint32_t pos = wcnt[w][dig] + (uint32_t)rank;
      if (pos < (uint32_t)n) {
        kout[pos] = key;
        vout[pos] = val;
      } else {
        atomicOr(d.status, kStatusInternal);  // a rank outside the sorted range: report, skip
      }
    }
    __syncthreads();
  }
}

// Per-tile [begin, end) from the sorted keys (range was zeroed beforehand).
__global__ void k_ranges(Dev d, const uint32_t* keys) {
  const int n = sort_count(d);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t key = keys[k];
    if (key >= (uint32_t)d.total_tiles) {
      atomicOr(d.status, kStatusInternal);
      continue;
    }
    if (k == 0 || keys[k - 1] != key) d.range[key].x = (uint32_t)k;
    if (k == n - 1 || keys[k + 1] != key) d.range[key].y = (uint32_t)(k + 1);
  }
}

cudaError_t launch_transform(const Dev& d, cudaStream_t s, bool zero_grad) {
  const int threads = 256, warps = threads / 32;
  k_transform<<<(d.n_elems + warps - 1) / warps, threads, 0, s>>>(d, zero_grad ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_scan(const Dev& d, cudaStream_t s) {
  k_scan<<<1, 1024, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_bin(const Dev& d, cudaStream_t s) {
  const int warps = 8;
  k_emit<<<(d.n_elems + warps - 1) / warps, warps * 32, 0, s>>>(d);
  const uint32_t* kin = d.keys0;
  const uint32_t* vin = d.vals0;
  for (int pass = 0; pass < d.n_sort_passes; ++pass) {
    uint32_t* kout = (pass & 1) ? d.keys0 : d.keys1;
    uint32_t* vout = (pass & 1) ? d.vals0 : d.vals1;
    const int shift = pass * kSortBits;
    k_sort_hist<<<d.sort_blocks, kSortThreads, 0, s>>>(d, shift, kin);
    k_sort_scan<<<1, 1024, 0, s>>>(d, d.sort_blocks);
    k_sort_scatter<<<d.sort_blocks, kSortThreads, 0, s>>>(d, shift, kin, vin, kout, vout);
    kin = kout;
    vin = vout;
  }
  cudaError_t e = cudaMemsetAsync(d.range, 0, sizeof(uint2) * (size_t)d.total_tiles, s);
  if (e != cudaSuccess) return e;
  k_ranges<<<256, 256, 0, s>>>(d, kin);
  return cudaGetLastError();
}

}  // namespace collage
