// Quality metrics of a collage (Sec. 6, "Metrics of Collage Quality", and the layout
// non-uniformity of the uniformity ablation, Sec. 6.1), computed on the device from a render pass
// at the current params.
//
// A pixel is object where O = 1 - Ihat >= 1/2, shape where the container coverage is >= 1/2, and
// overlap where at least two elements have sd >= 0 (c_i >= 1/2).  Per problem: LC = object pixels
// inside the shape / shape pixels, OO = overlap pixels / shape pixels, EA = object pixels outside
// the shape / shape pixels, and L-nU = the mean, over the non-object shape pixels, of the squared
// distance (unit coordinates) from the pixel centre to the nearest object pixel centre.  All
// counts and squared distances are integers, summed exactly.
#include "collage.h"
#include "internal.h"

namespace collage {

constexpr int kMetWarps = 4;
constexpr int kMetFar = 1 << 20;  // "no object pixel in this column" (rows)

// Counts per problem: cnt[4p + 0] object in shape, [1] shape, [2] overlap, [3] object outside the
// shape; obj[pix] = 1 for an object pixel.  One tile per warp.
template <int T>
__global__ void __launch_bounds__(kMetWarps * 32) k_metric_counts(Dev d, uint8_t* obj, unsigned long long* cnt) {
  constexpr int NP = T * T, PPL = NP / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int tile = blockIdx.x * kMetWarps + wid; tile < d.total_tiles; tile += gridDim.x * kMetWarps) {
    int p = 0, lo = 0, hi = d.n_probs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (d.prob_tile_base[mid] <= tile) lo = mid;
      else hi = mid - 1;
    }
    p = lo;
    const int lt = tile - d.prob_tile_base[p], ntx = d.prob_ntx[p], res = d.prob_res[p];
    const int tx = lt % ntx, ty = lt / ntx;
    const long long pixbase = d.prob_pix_base[p];
    const int m = d.tile_m[tile];
    const int* slots = d.tile_sorted_slot + (size_t)tile * d.tile_cap;
    unsigned c_in = 0, c_shape = 0, c_over = 0, c_out = 0;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int local = lane + 32 * k;
      const int X = tx * T + local % T, Y = ty * T + local / T;
      bool valid = X < res && Y < res, o = false, sh = false, ov = false;
      if (valid) {
        const long long pix = pixbase + (long long)Y * res + X;
        int n_in = 0;
        for (int i = 0; i < m && n_in < 2; ++i) {
          const int sl = slots[i];
          const uint8_t cls = d.pair_cls[sl];
          if (cls == kPairIn) n_in += 1;
          else if (cls == kPairNear && d.saved[(size_t)sl * NP + local].x >= 0.0f) n_in += 1;
        }
        o = d.img_I[pix] <= 0.5f;
        sh = d.covc[pix] >= 0.5f;
        ov = n_in >= 2;
        obj[pix] = o ? 1 : 0;
      }
      c_in += __popc(__ballot_sync(0xffffffffu, o && sh));
      c_shape += __popc(__ballot_sync(0xffffffffu, sh));
      c_over += __popc(__ballot_sync(0xffffffffu, ov));
      c_out += __popc(__ballot_sync(0xffffffffu, o && !sh));
    }
    if (lane == 0) {
      if (c_in) atomicAdd(&cnt[4 * p + 0], (unsigned long long)c_in);
      if (c_shape) atomicAdd(&cnt[4 * p + 1], (unsigned long long)c_shape);
      if (c_over) atomicAdd(&cnt[4 * p + 2], (unsigned long long)c_over);
      if (c_out) atomicAdd(&cnt[4 * p + 3], (unsigned long long)c_out);
    }
  }
}

// Column pass of the distance transform: rows to the nearest object pixel of the same column.
__global__ void k_metric_cols(Dev d, const uint8_t* obj, int* gcol, int max_res) {
  const int p = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  const int res = d.prob_res[p];
  if (k >= res || k >= max_res) return;
  const long long pb = d.prob_pix_base[p];
  int last = -kMetFar;
  for (int i = 0; i < res; ++i) {
    const long long pix = pb + (long long)i * res + k;
    if (obj[pix]) last = i;
    gcol[pix] = last > -kMetFar ? i - last : kMetFar;
  }
  last = kMetFar + res;
  for (int i = res - 1; i >= 0; --i) {
    const long long pix = pb + (long long)i * res + k;
    if (obj[pix]) last = i;
    if (last - i < gcol[pix]) gcol[pix] = last - i;
  }
}

// Row pass, one row per warp: for each non-object shape pixel the squared distance to the nearest
// object pixel is the minimum over the columns k of (j - k)^2 + gcol(i, k)^2; the sum over the
// row goes to sums[p] (exact 64-bit integers).
__global__ void __launch_bounds__(kMetWarps * 32) k_metric_rows(Dev d, const uint8_t* obj, const int* gcol,
                                                              unsigned long long* sums, int max_res) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int p = blockIdx.y, i = blockIdx.x * kMetWarps + wid;
  const int res = d.prob_res[p];
  if (i >= res || i >= max_res) return;
  const long long rowb = d.prob_pix_base[p] + (long long)i * res;
  unsigned long long acc = 0;
  for (int j = lane; j < res; j += 32) {
    if (obj[rowb + j] || !(d.covc[rowb + j] >= 0.5f)) continue;
    long long best = (long long)kMetFar * kMetFar;
    for (int k = 0; k < res; ++k) {
      const long long g = gcol[rowb + k];
      const long long dj = j - k;
      const long long d2 = dj * dj + g * g;
      best = d2 < best ? d2 : best;
    }
    if (best < (long long)kMetFar * kMetFar) acc += (unsigned long long)best;
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0 && acc) atomicAdd(&sums[p], acc);
}

cudaError_t launch_metrics(const Dev& d, cudaStream_t s, uint8_t* obj, int* gcol,
                           unsigned long long* cnt, unsigned long long* sums, int max_res) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 4 * d.n_probs, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * d.n_probs, s);
  if (e != cudaSuccess) return e;
  const int tgrid = (d.total_tiles + kMetWarps - 1) / kMetWarps;
  if (d.tile == 8) k_metric_counts<8><<<tgrid, kMetWarps * 32, 0, s>>>(d, obj, cnt);
  else if (d.tile == 16) k_metric_counts<16><<<tgrid, kMetWarps * 32, 0, s>>>(d, obj, cnt);
  else return cudaErrorInvalidValue;
  k_metric_cols<<<dim3((max_res + 127) / 128, d.n_probs), 128, 0, s>>>(d, obj, gcol, max_res);
  k_metric_rows<<<dim3((max_res + kMetWarps - 1) / kMetWarps, d.n_probs), kMetWarps * 32, 0, s>>>(
      d, obj, gcol, sums, max_res);
  return cudaGetLastError();
}

}  // namespace collage
