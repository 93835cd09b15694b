// Skeleton-based initialisation (Sec. 4.1): the medial axis of the container and its medial width
// (distance to the nearest boundary point), then the elements placed along the axis, larger ones
// where the width is larger.
//
// On the container raster of the current level (inside: coverage >= 1/2; the pixels one step beyond
// the image count as outside):
//  - D2(p): the squared distance, in pixels, from an inside pixel centre to the nearest outside pixel
//    centre (exact integers: a column pass, then per row the minimum over columns k of
//    (j - k)^2 + g(k)^2);
//  - the medial axis: the ridge of D2, the inside pixels that are a maximum of D2 along one of the
//    four lines through them (horizontal, vertical, the two diagonals): D2 >= both line neighbours
//    and > at least one (neighbours beyond the image count 0);
//  - placement, per problem: the elements in decreasing radius r = rbin s res (pixels; ties: lower
//    index first) each take the axis pixel of largest D2 (ties: lower pixel index) whose clearance
//    min_j (|p - c_j| - r_j) over the elements placed so far is >= r; if no axis pixel has that
//    clearance, the one of largest clearance.  Clearances are float32 with a fixed operation order,
//    so every decision is reproducible.  The element's translation becomes its pixel centre;
//    rotation and scale are kept.
#include <cfloat>
#include <cooperative_groups.h>

#include "collage.h"
#include "internal.h"

namespace collage {

namespace cg = cooperative_groups;

constexpr int kMatWarps = 4;
constexpr int kPlaceThreads = 512;
constexpr int kPlaceCluster = 8;  // blocks (one thread-block cluster) per problem

__device__ __forceinline__ bool inside_px(const Dev& d, long long pix) { return d.covc[pix] >= 0.5f; }

// Column pass: rows to the nearest outside pixel of the same column (rows -1 and res are outside).
__global__ void k_mat_cols(Dev d, int* gcol, int max_res) {
  const int p = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  const int res = d.prob_res[p];
  if (k >= res || k >= max_res) return;
  const long long pb = d.prob_pix_base[p];
  // rows in groups of 8 whose coverages are read together (the loads are independent; only the
  // running index of the last outside pixel carries from row to row)
  constexpr int G = 8;
  int last = -1;
  for (int i0 = 0; i0 < res; i0 += G) {
    bool out[G];
#pragma unroll
    for (int u = 0; u < G; ++u) out[u] = i0 + u < res && !inside_px(d, pb + (long long)(i0 + u) * res + k);
#pragma unroll
    for (int u = 0; u < G; ++u) {
      if (i0 + u >= res) break;
      if (out[u]) last = i0 + u;
      gcol[pb + (long long)(i0 + u) * res + k] = i0 + u - last;
    }
  }
  last = res;
  for (int i1 = res - 1; i1 >= 0; i1 -= G) {
    bool out[G];
    int g[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int i = i1 - u;
      out[u] = i >= 0 && !inside_px(d, pb + (long long)i * res + k);
      g[u] = i >= 0 ? gcol[pb + (long long)i * res + k] : 0;
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int i = i1 - u;
      if (i < 0) break;
      if (out[u]) last = i;
      if (last - i < g[u]) gcol[pb + (long long)i * res + k] = last - i;
    }
  }
}

// Row pass, one row per warp: D2 = min over the columns k in [-1, res] of (j - k)^2 + g(k)^2, with
// g = 0 in the two columns beyond the image; 0 for outside pixels.
__global__ void __launch_bounds__(kMatWarps * 32) k_mat_rows(Dev d, const int* gcol, unsigned* d2,
                                                             int max_res) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int p = blockIdx.y, i = blockIdx.x * kMatWarps + wid;
  const int res = d.prob_res[p];
  if (i >= res || i >= max_res) return;
  const long long rowb = d.prob_pix_base[p] + (long long)i * res;
  for (int j = lane; j < res; j += 32) {
    if (!inside_px(d, rowb + j)) {
      d2[rowb + j] = 0u;
      continue;
    }
    long long best = (long long)(j + 1) * (j + 1);
    const long long right = (long long)(res - j) * (res - j);
    if (right < best) best = right;
    for (int k = 0; k < res; ++k) {
      const long long g = gcol[rowb + k], dj = j - k;
      const long long v = dj * dj + g * g;
      best = v < best ? v : best;
    }
    d2[rowb + j] = (unsigned)best;
  }
}

// Medial axis test per pixel; the axis pixels are appended to their problem's candidate list
// (in no particular order: the placement orders them by key).
__global__ void k_mat_axis(Dev d, const unsigned* d2, int* cand, int* n_cand, int* axis_out,
                           float* width_out) {
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= d.total_pix) return;
  int p = 0, lo = 0, hi = d.n_probs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d.prob_pix_base[mid] <= pix) lo = mid;
    else hi = mid - 1;
  }
  p = lo;
  const long long pb = d.prob_pix_base[p];
  const int res = d.prob_res[p];
  const int local = (int)(pix - pb), y = local / res, x = local % res;
  const unsigned a = d2[pix];
  auto at = [&](int xx, int yy) -> unsigned {
    return xx < 0 || yy < 0 || xx >= res || yy >= res ? 0u : d2[pb + (long long)yy * res + xx];
  };
  bool axis = false;
  if (a > 0) {
    const int dirs[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};
    for (int k = 0; k < 4 && !axis; ++k) {
      const unsigned u = at(x + dirs[k][0], y + dirs[k][1]), v = at(x - dirs[k][0], y - dirs[k][1]);
      axis = a >= u && a >= v && (a > u || a > v);
    }
  }
  if (axis) cand[pb + atomicAdd(&n_cand[p], 1)] = local;
  if (axis_out) axis_out[pix] = axis ? 1 : 0;
  if (width_out) width_out[pix] = a > 0 ? sqrtf((float)a) : 0.0f;
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long* s) {
  for (int o = 16; o; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  __syncthreads();  // the previous reduction's readers are done
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0ull;
    for (int o = 16; o; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (threadIdx.x == 0) s[0] = v;
  }
  __syncthreads();
  return s[0];
}

// The block's maxima of two keys in one reduction.
__device__ __forceinline__ void block_max2(unsigned long long& a, unsigned long long& b, unsigned long long (*s)[2]) {
  for (int o = 16; o; o >>= 1) {
    const unsigned long long wa = __shfl_xor_sync(0xffffffffu, a, o);
    const unsigned long long wb = __shfl_xor_sync(0xffffffffu, b, o);
    a = wa > a ? wa : a;
    b = wb > b ? wb : b;
  }
  __syncthreads();  // the previous reduction's readers are done
  if ((threadIdx.x & 31) == 0) {
    s[threadIdx.x >> 5][0] = a;
    s[threadIdx.x >> 5][1] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool in = threadIdx.x < (blockDim.x >> 5);
    a = in ? s[threadIdx.x][0] : 0ull;
    b = in ? s[threadIdx.x][1] : 0ull;
    for (int o = 16; o; o >>= 1) {
      const unsigned long long wa = __shfl_xor_sync(0xffffffffu, a, o);
      const unsigned long long wb = __shfl_xor_sync(0xffffffffu, b, o);
      a = wa > a ? wa : a;
      b = wb > b ? wb : b;
    }
  }
}

// A float's bits as an unsigned key with the float's order (negative values included).
__device__ __forceinline__ unsigned ordered(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Greedy placement, one thread-block cluster of kPlaceCluster blocks per problem.  Block 0 first
// ranks the elements by radius (ties: lower index) into order[]; every block then gathers its
// share of the axis pixels (D2, packed coordinates, clearance) into dynamic shared memory (else
// into cand, gxy and clear); each step is one pass of every block over its share: the clearances
// take the previous element's disk into account and the block reduces its two candidates (the
// widest pixel with room, the pixel of largest clearance); after one cluster barrier every block
// reads the cluster's partials from the blocks' shared memory (double-buffered by step parity, so
// one barrier a step suffices) and takes the same choice; block 0 writes the translation.  Every
// block runs the same steps and barriers, and a last barrier keeps each block's shared memory
// alive until the others have read it.
constexpr int kPlaceRankMax = 4096;                // elements ranked in shared memory (more: a
                                                   // reduction per step)
constexpr int kPlaceSmemCandBytes = 160 * 1024;    // candidates of a placement block (D2,
constexpr int kPlaceSmemCands = kPlaceSmemCandBytes / 12;  // coordinates, clearance)
// then, for the ranked elements, each step's element and radius
constexpr int kPlaceSmem = kPlaceSmemCandBytes + kPlaceRankMax * 8;
static_assert(kPlaceSmemCandBytes >= kPlaceRankMax * 8, "the ranking keys share the candidates' space");

__device__ __forceinline__ unsigned long long elem_key(const Dev& d, int e, float fres) {
  const float r = __fmul_rn(__fmul_rn(d.elem_rbin[e], d.q[e].w), fres);
  return ((unsigned long long)__float_as_uint(r) << 32) | (0xffffffffu - (unsigned)e);
}

__global__ void __launch_bounds__(kPlaceThreads) k_mat_place(Dev d, int* cand, const int* n_cand,
                                                             const unsigned* d2, float* clear, int* gxy,
                                                             int* order) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ unsigned long long s_red[kPlaceThreads / 32];
  __shared__ unsigned long long s_red2[kPlaceThreads / 32][2];
  __shared__ unsigned long long s_part[2][2];  // per step parity: (widest with room, largest clearance)
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int p = blockIdx.x / kPlaceCluster;
  const int res = d.prob_res[p], nc = n_cand[p];
  const long long pb = d.prob_pix_base[p];
  const int e0 = d.prob_elem_base[p], e1 = d.prob_elem_base[p + 1], ne = e1 - e0;
  if (nc == 0) return;  // no inside pixel: the params stay (every block of the cluster leaves here)
  const float fres = (float)res;
  // the elements in placement order: decreasing key (radius bits, then the lower index)
  const bool ranked = ne <= kPlaceRankMax;
  if (rank == 0) {
    if (ranked) {
      unsigned long long* s_key = reinterpret_cast<unsigned long long*>(s_dyn);
      for (int i = threadIdx.x; i < ne; i += kPlaceThreads) s_key[i] = elem_key(d, e0 + i, fres);
      __syncthreads();
      for (int i = threadIdx.x; i < ne; i += kPlaceThreads) {
        const unsigned long long k = s_key[i];
        int rnk = 0;
        for (int j = 0; j < ne; ++j) rnk += s_key[j] > k ? 1 : 0;
        order[e0 + rnk] = e0 + i;
      }
    } else {
      for (int i = threadIdx.x; i < ne; i += kPlaceThreads) order[e0 + i] = 0;  // 0: not placed yet
    }
    __threadfence();
  }
  cluster.sync();  // order[] is complete (and block 0's keys' space is free)
  int* s_ord = reinterpret_cast<int*>(s_dyn + kPlaceSmemCandBytes);
  float* s_rad = reinterpret_cast<float*>(s_dyn + kPlaceSmemCandBytes + 4 * kPlaceRankMax);
  if (ranked)
    for (int i = threadIdx.x; i < ne; i += kPlaceThreads) {
      const int e = order[e0 + i];
      s_ord[i] = e;
      s_rad[i] = __fmul_rn(__fmul_rn(d.elem_rbin[e], d.q[e].w), fres);
    }
  // this block's share of the candidates: D2, x | y << 16, the clearance
  const int c_lo = (int)((long long)nc * rank / kPlaceCluster);
  const int mc = (int)((long long)nc * (rank + 1) / kPlaceCluster) - c_lo;
  const bool in_smem = mc <= kPlaceSmemCands;
  unsigned* cd2 = in_smem ? reinterpret_cast<unsigned*>(s_dyn) : reinterpret_cast<unsigned*>(cand + pb + c_lo);
  int* cxy = in_smem ? reinterpret_cast<int*>(s_dyn + 4 * kPlaceSmemCands) : gxy + pb + c_lo;
  float* ccl = in_smem ? reinterpret_cast<float*>(s_dyn + 8 * kPlaceSmemCands) : clear + pb + c_lo;
  for (int c = threadIdx.x; c < mc; c += kPlaceThreads) {
    const int idx = cand[pb + c_lo + c];
    const unsigned w = d2[pb + idx];
    cd2[c] = w;
    cxy[c] = (idx % res) | ((idx / res) << 16);
    ccl[c] = FLT_MAX;
  }
  __syncthreads();
  int px = 0, py = 0;  // the previous element's pixel and radius (none before the first step)
  float pr = -1.0f;
  for (int step = 0; step < ne; ++step) {
    int e;
    float r;
    if (ranked) {
      e = s_ord[step];
      r = s_rad[step];
    } else {  // the largest element not yet placed, by a reduction (the same in every block)
      unsigned long long ek = 0;
      for (int i = threadIdx.x; i < ne; i += kPlaceThreads) {
        if (order[e0 + i]) continue;
        const unsigned long long k = elem_key(d, e0 + i, fres);
        ek = k > ek ? k : ek;
      }
      ek = block_max(ek, s_red);
      e = (int)(0xffffffffu - (unsigned)(ek & 0xffffffffu));
      r = __fmul_rn(__fmul_rn(d.elem_rbin[e], d.q[e].w), fres);
    }
    // one pass: the previous element's disk into the clearances, then the widest axis pixel with
    // clearance >= r (key: D2, then the lower pixel index), and the largest clearance as fallback
    unsigned long long ck = 0, fk = 0;
    for (int c = threadIdx.x; c < mc; c += kPlaceThreads) {
      const int xy = cxy[c], x = xy & 0xffff, y = xy >> 16;
      float cl = ccl[c];
      if (pr >= 0.0f) {
        const int dx = x - px, dy = y - py;
        const float dist = __fsub_rn(sqrtf(__int2float_rn(dx * dx + dy * dy)), pr);
        if (dist < cl) {
          cl = dist;
          ccl[c] = cl;
        }
      }
      const unsigned long long low = 0xffffffffu - (unsigned)(y * res + x);
      if (cl >= r) {
        const unsigned long long k = ((unsigned long long)cd2[c] << 32) | low;
        ck = k > ck ? k : ck;
      }
      const unsigned long long kf = ((unsigned long long)ordered(cl) << 32) | low;
      fk = kf > fk ? kf : fk;
    }
    block_max2(ck, fk, s_red2);
    if (threadIdx.x == 0) {
      s_part[step & 1][0] = ck;
      s_part[step & 1][1] = fk;
    }
    cluster.sync();  // every block's partials of this step are written
    // every warp reduces the cluster's partials itself (lane k reads block k's)
    unsigned long long a = 0, b = 0;
    const int lane = threadIdx.x & 31;
    if (lane < kPlaceCluster) {
      const unsigned long long* part = cluster.map_shared_rank(&s_part[step & 1][0], (unsigned)lane);
      a = part[0];
      b = part[1];
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long wa = __shfl_xor_sync(0xffffffffu, a, o);
      const unsigned long long wb = __shfl_xor_sync(0xffffffffu, b, o);
      a = wa > a ? wa : a;
      b = wb > b ? wb : b;
    }
    const unsigned long long best = a != 0 ? a : b;  // none has room: the largest clearance
    const int idx = (int)(0xffffffffu - (unsigned)(best & 0xffffffffu));
    px = idx % res;
    py = idx / res;
    pr = r;
    if (threadIdx.x == 0) {
      if (!ranked) order[e] = 1;  // (every block marks it: its own next reduction reads it)
      if (rank == 0) {
        float4 q = d.q[e];
        q.x = __fdiv_rn(__fadd_rn((float)px, 0.5f), fres);
        q.y = __fdiv_rn(__fadd_rn((float)py, 0.5f), fres);
        d.q[e] = q;
      }
    }
    // the unranked flags are visible to the next reduction (the partials' buffer of this step is
    // not written again before the next step's cluster barrier, which every thread passes)
    if (!ranked) __syncthreads();
  }
  cluster.sync();  // no block leaves while another may still read its partials
}

cudaError_t launch_mat_init(const Dev& d, cudaStream_t s, int max_res, int* gcol, unsigned* d2,
                            int* cand, int* n_cand, float* clear, int* order, int* axis_out,
                            float* width_out) {
  cudaError_t e = cudaMemsetAsync(n_cand, 0, sizeof(int) * d.n_probs, s);
  if (e != cudaSuccess) return e;
  k_mat_cols<<<dim3((max_res + 127) / 128, d.n_probs), 128, 0, s>>>(d, gcol, max_res);
  k_mat_rows<<<dim3((max_res + kMatWarps - 1) / kMatWarps, d.n_probs), kMatWarps * 32, 0, s>>>(
      d, gcol, d2, max_res);
  const long long np = d.total_pix;
  k_mat_axis<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(d, d2, cand, n_cand, axis_out, width_out);
  // gcol is free after the row pass: it holds the candidates' coordinates when they do not fit in
  // shared memory
  e = cudaFuncSetAttribute(k_mat_place, cudaFuncAttributeMaxDynamicSharedMemorySize, kPlaceSmem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(d.n_probs * kPlaceCluster);
  cfg.blockDim = dim3(kPlaceThreads);
  cfg.dynamicSmemBytes = kPlaceSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kPlaceCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mat_place, d, cand, n_cand, d2, clear, gcol, order);
}

}  // namespace collage
