// Transform (Eq. 2) and tile binning.
//
// Binning is a counting sort keyed on the tile: the transform kernel counts, per tile, the elements
// whose tile rectangle covers it (integer atomics); one prefix scan over the tiles turns the counts
// into [begin, end) ranges; emission places each (tile, element) pair in its tile's range (and
// counts the tile back down to zero for the next iteration); the raster kernel then orders each
// tile's short list by element id before using it, so every tile lists its elements in increasing
// order whatever the order of the atomics.  The tile rectangle follows a fixed float formula
// (bin_rect), so the bins are bit-exact against the oracle's rule.
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

// Vertex of an element relative to its translation, in pixels: R(theta) (s v) * res, formed in
// double and rounded once.  A segment's end point and the next segment's start point come from the
// same call, so they are bitwise equal (the winding test relies on it).
__device__ __forceinline__ float2 vertex_px(const float2 v, double c, double sn, double sc) {
  const double x = sc * (c * (double)v.x - sn * (double)v.y);
  const double y = sc * (sn * (double)v.x + c * (double)v.y);
  return make_float2((float)x, (float)y);
}

// One warp per element: segment records (start, direction, end y, 1/|e|^2), translation in pixels
// as a float hi/lo pair, outline box grown by the coverage margin, tile rectangle, and the
// per-tile element counts of the counting sort.
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
  const int v0 = d.elem_voff[g], v1 = d.elem_voff[g + 1], nv = v1 - v0;
  const bool closed = d.elem_closed[g] != 0;
  float xmin = FLT_MAX, ymin = FLT_MAX, xmax = -FLT_MAX, ymax = -FLT_MAX;
  for (int k = lane; k < nv; k += 32) {
    const float2 a = vertex_px(d.vloc[v0 + k], c, sn, sc);
    xmin = fminf(xmin, a.x);
    xmax = fmaxf(xmax, a.x);
    ymin = fminf(ymin, a.y);
    ymax = fmaxf(ymax, a.y);
    float4 sa = make_float4(a.x, a.y, 0.f, 0.f);
    float2 sb = make_float2(a.y, 0.f);
    if (closed || k + 1 < nv) {
      const float2 b = vertex_px(d.vloc[v0 + (k + 1 == nv ? 0 : k + 1)], c, sn, sc);
      const float ex = b.x - a.x, ey = b.y - a.y, ee = ex * ex + ey * ey;
      sa.z = ex;
      sa.w = ey;
      sb = make_float2(b.y, ee > 0.0f ? 1.0f / ee : 0.0f);
    }
    d.segA[v0 + k] = sa;
    d.segB[v0 + k] = sb;
  }
  xmin = warp_min(xmin);
  ymin = warp_min(ymin);
  xmax = warp_max(xmax);
  ymax = warp_max(ymax);
  int4 r = make_int4(0, 0, -1, -1);
  if (lane == 0) {
    const double tx = (double)q.x * res, ty = (double)q.y * res;
    const float hx = (float)tx, hy = (float)ty;
    d.tpx[g] = make_float4(hx, hy, (float)(tx - (double)hx), (float)(ty - (double)hy));
    const float hw = closed ? 0.0f : d.elem_hw[g];
    // outline box relative to the translation, grown by the coverage margin (+ rounding slack)
    const float m = d.L.rho_px + d.L.pad_px + hw * (float)res + 0.01f;
    d.bbox[g] = make_float4(xmin - m, ymin - m, xmax + m, ymax + m);
    const bool finite = isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w) && q.w > 0.0f;
    if (finite) r = bin_rect(q, d.elem_rbin[g], hw, res, d.tile, d.L.rho_px, d.L.pad_px);
    else atomicOr(d.status, kStatusBadParam);
    d.rect[g] = r;
    if (zero_grad) d.dq[g] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  r.x = __shfl_sync(0xffffffffu, r.x, 0);
  r.y = __shfl_sync(0xffffffffu, r.y, 0);
  r.z = __shfl_sync(0xffffffffu, r.z, 0);
  r.w = __shfl_sync(0xffffffffu, r.w, 0);
  if (r.z < r.x || r.w < r.y) return;
  const int w = r.z - r.x + 1, n = w * (r.w - r.y + 1);
  const int tb = d.prob_tile_base[p], ntx = d.prob_ntx[p];
  for (int i = lane; i < n; i += 32) atomicAdd(&d.tile_cnt[tb + (r.y + i / w) * ntx + r.x + i % w], 1);
}

// Exclusive scan of the per-tile counts into [begin, end) ranges (one block; a contiguous chunk
// per thread).  The total is the pair count; above the capacity the overflow bit is latched.
__global__ void __launch_bounds__(1024) k_tile_scan(Dev d) {
  __shared__ int wsum[32];
  const int n = d.total_tiles, t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = min(t * per, n), e = min(b + per, n);
  int s = 0;
  for (int i = b; i < e; ++i) s += d.tile_cnt[i];
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
    const int c = d.tile_cnt[i];
    d.range[i] = make_uint2((uint32_t)run, (uint32_t)(run + c));
    run += c;
  }
  if (t == 1023) {
    *d.total_pairs = run;
    if (run > d.cap) atomicOr(d.status, kStatusOverflow);
  }
}

// Emission: each (tile, element) pair takes a slot of its tile's range by counting the tile back
// down (so the counts are zero again for the next iteration, also after an overflow).
__global__ void k_emit(Dev d) {
  const int g = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= d.n_elems) return;
  const int4 r = d.rect[g];
  if (r.z < r.x || r.w < r.y) return;
  const int w = r.z - r.x + 1, n = w * (r.w - r.y + 1);
  const int p = d.elem_prob[g];
  const int tb = d.prob_tile_base[p], ntx = d.prob_ntx[p];
  for (int i = lane; i < n; i += 32) {
    const int t = tb + (r.y + i / w) * ntx + r.x + i % w;
    const int slot = atomicSub(&d.tile_cnt[t], 1) - 1;
    const unsigned pos = d.range[t].x + (unsigned)slot;
    if (pos < (unsigned)d.cap) d.pair_elem[pos] = g;
  }
}

cudaError_t launch_transform(const Dev& d, cudaStream_t s, bool zero_grad) {
  const int threads = 256, warps = threads / 32;
  k_transform<<<(d.n_elems + warps - 1) / warps, threads, 0, s>>>(d, zero_grad ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_scan(const Dev& d, cudaStream_t s) {
  k_tile_scan<<<1, 1024, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_bin(const Dev& d, cudaStream_t s) {
  const int warps = 8;
  k_emit<<<(d.n_elems + warps - 1) / warps, warps * 32, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace collage
