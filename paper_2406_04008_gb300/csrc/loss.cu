// Even-distribution term (Eq. 7), loss assembly (Eq. 8), the deterministic gradient reduction and
// the flush of a pending Adam step.
//
// Eq. 7 as implemented: K box kernels of widths 5 + 6k pixels (k = 0..K-1) dilate the occupancy
// O = 1 - Ihat; D_k = min(1, B_k) with B_k the zero-padded box sum; the term sums
// w_k M_C (1 - O) (1 - D_k) over the container.  Its adjoint is
//   dL_u/dO(q) = sum_k w_k [ -M_C(q)(1 - D_k(q)) - sum_{p in box_k(q)} M_C(p)(1 - O(p)) [B_k(p) < 1] ].
// Both passes stage a 32 x 32 tile plus a halo of the largest radius in shared memory and form the
// box sums in fixed point: the forward pass from one integral image of the staged occupancy, the
// adjoint (whose summand differs per kernel) separably, rows then columns, with running windows.
#include "internal.h"

namespace collage {

constexpr int kDT = 32;       // dilation tile side
constexpr int kDThreads = 256;

__device__ __forceinline__ int find_prob_d(const int* base, int P, int t) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Box sums in fixed point: a value v in [0, 1] is held as round(v 2^Q) in a 32-bit unsigned
// integer, with Q the largest precision for which (w^2 + w) 2^Q < 2^32, w the widest kernel (so a
// full box, w^2 2^Q, may pass 2^31).  Integer sums are exact in any order: unsigned wrap-around
// cancels between the add and the subtract of a running window, and in the four-corner difference
// of an integral image, since every box sum is below 2^32.  The adjoint slides one window along
// kSeg outputs of a row (or column) of one kernel, with one add and one subtract per output and no
// rounding drift; the forward pass reads every kernel's box sums from one integral image.  The
// kernels are instantiated per number of dilations K so that every window loop unrolls.
//
// Shared-memory layout, chosen so that the 32 lanes of a warp touch 32 distinct banks: the staged
// region and the integral image have odd row strides; the horizontal sums H of kernel k keep only
// the 32 + 2 r_k rows its vertical pass reads, with a row stride of 33; consecutive lanes take
// consecutive rows in the horizontal pass and the row scan, and consecutive columns in the
// vertical pass, the column scan and the staging.
constexpr int kSeg = 32;  // one running window per row of the tile
constexpr int kNSeg = kDT / kSeg;
constexpr int kHP = kDT + 1;  // row stride of H
constexpr int kFlagOwn = 1;   // container coverage is nonzero somewhere on the tile
constexpr int kFlagHalo = 2;  // ... or somewhere within the halo of the largest kernel

__host__ __device__ constexpr int dil_r(int k) { return 2 + 3 * k; }  // (5 + 6k - 1) / 2
__host__ __device__ constexpr int hrows(int k) { return kDT + 2 * dil_r(k); }
__host__ __device__ constexpr int hbase(int k) { return k == 0 ? 0 : hbase(k - 1) + hrows(k - 1); }
__host__ __device__ constexpr int qbits(int w) {  // at most 23: bits 24..31 carry the B_k < 1 mask
  int q = 0;
  while (q < 23 && ((unsigned long long)(w * w + w) << (q + 1)) < (1ull << 32)) ++q;
  return q;
}

template <int K>
struct DilGeom {
  static constexpr int h = dil_r(K - 1);  // radius of the widest kernel
  static constexpr int S = kDT + 2 * h;   // staged side
  static constexpr int SP = S | 1;        // staged row stride (odd)
  static constexpr int HR = hbase(K);     // rows of H over all kernels
  static constexpr int Q = qbits(2 * h + 1);
  static constexpr int CW = S <= 32 ? 32 : S <= 64 ? 64 : 128;  // staging: threads per staged row
  static_assert(CW <= kDThreads, "a staged row fits the block");
};

template <int K>
__device__ __forceinline__ uint32_t to_fixed(float v) {
  return __float2uint_rn(v * (float)(1u << DilGeom<K>::Q));
}

// One horizontal running-window item of kernel k: outputs c0..c0+kSeg-1 of staged row
// rr = h - r + li, H[k][li][c] = sum_{|dc| <= r_k} src(k, rr, c + h + dc).
template <int K, int k, class Src>
__device__ __forceinline__ void hsum_one(const Src& src, uint32_t* H, int it) {
  constexpr int h = DilGeom<K>::h, r = dil_r(k), rows = hrows(k);
  const int li = it % rows, seg = it / rows, rr = h - r + li;
  const int c0 = seg * kSeg;
  uint32_t acc = 0u;
#pragma unroll
  for (int dc = -r; dc <= r; ++dc) acc += src(k, rr, c0 + h + dc);
  uint32_t* out = H + (hbase(k) + li) * kHP + c0;
  out[0] = acc;
#pragma unroll
  for (int c = 1; c < kSeg; ++c) {
    acc += src(k, rr, c0 + c + h + r) - src(k, rr, c0 + c + h - r - 1);
    out[c] = acc;
  }
}

// Vertical pass fused with the per-pixel output: a thread forms the box sums of all K kernels at
// kVRows consecutive output rows of one column (a running window per kernel), then uses them
// directly, so no per-kernel result image is kept in shared memory.
// B[k][i] = sum_{|dr| <= r_k} H[k][r0 + i + r_k + dr][c].
constexpr int kVRows = 4;
constexpr int kVItems = kDT * (kDT / kVRows);
static_assert(kVItems == kDThreads, "one output item per thread");

template <int K, int k = 0>
__device__ __forceinline__ void vsums_col(const uint32_t* H, int c, int r0, uint32_t (&B)[K][kVRows]) {
  if constexpr (k < K) {
    constexpr int r = dil_r(k);
    const uint32_t* col = H + hbase(k) * kHP + c;
    uint32_t acc = 0u;
#pragma unroll
    for (int j = 0; j <= 2 * r; ++j) acc += col[(r0 + j) * kHP];
    B[k][0] = acc;
#pragma unroll
    for (int i = 1; i < kVRows; ++i) {
      acc += col[(r0 + i + 2 * r) * kHP] - col[(r0 + i - 1) * kHP];
      B[k][i] = acc;
    }
    vsums_col<K, k + 1>(H, c, r0, B);
  }
}

// Item `it` of the flattened list of all kernels' horizontal items: every thread of the block
// gets work, whatever the kernel sizes.
template <int K, int k = 0, class Src>
__device__ __forceinline__ void hsum_item(const Src& src, uint32_t* H, int it) {
  if constexpr (k < K) {
    constexpr int items_k = hrows(k) * kNSeg;
    if (it < items_k) hsum_one<K, k>(src, H, it);
    else hsum_item<K, k + 1>(src, H, it - items_k);
  }
}

struct OccSrc {  // occupancy O of the staged region, the same for every kernel
  const uint32_t* sO;
  int SP;
  __device__ uint32_t operator()(int, int rr, int cc) const { return sO[rr * SP + cc]; }
};

struct GSrc {  // G_k = M_C (1 - O) where B_k < 1, else 0; the staged word holds the fixed-point
               // M_C (1 - O) in bits 0..23 and the B_k < 1 bits from bit 24 on (one load per use)
  const uint32_t* sM;
  int SP;
  __device__ uint32_t operator()(int k, int rr, int cc) const {
    const uint32_t x = sM[rr * SP + cc];
    // bit 24 + k moved to the sign and spread over the word: all ones where B_k < 1
    return x & 0xffffffu & (uint32_t)((int)(x << (7 - k)) >> 31);
  }
};

template <int K, class Src>
__device__ __forceinline__ void hsums_all(const Src& src, uint32_t* H) {
  for (int it = threadIdx.x; it < DilGeom<K>::HR * kNSeg; it += blockDim.x) hsum_item<K>(src, H, it);
}

__device__ __forceinline__ int dil_flags(const Dev& d, int dt) {
  return d.dtile_flags ? (int)d.dtile_flags[dt] : (kFlagOwn | kFlagHalo);
}

// The tiles a pass visits: those with the given flag, from the per-level list (every tile when
// there is no list).  Tiles off the list hold zeros written once per level.
__device__ __forceinline__ int dil_count(const Dev& d, int which) {
  return d.dtile_list ? d.dtile_n[which] : d.total_dtiles;
}
__device__ __forceinline__ int dil_tile(const Dev& d, int which, int i) {
  return d.dtile_list ? d.dtile_list[which * d.total_dtiles + i] : i;
}

// The forward pass forms every box sum from one integral image of the staged occupancy:
// II[i][j] = sum of the staged values at rows < i and columns < j (row 0 and column 0 are zero), so
// B_k at a pixel is four loads at offsets fixed by r_k.  Unsigned wrap-around is exact here too.
template <int K>
struct IIGeom {
  static constexpr int S = DilGeom<K>::S;
  static constexpr int P = S + 1;  // row stride and side of II; odd, as S is even
  static_assert(P % 2 == 1, "odd row stride");
};

template <int K>
__global__ void __launch_bounds__(kDThreads, 5) k_dilate_fwd(Dev d) {
  pdl_enter();
  constexpr int S = DilGeom<K>::S, P = IIGeom<K>::P, h = DilGeom<K>::h, Q = DilGeom<K>::Q;
  constexpr float inv_q = 1.0f / (float)(1u << Q);
  extern __shared__ uint32_t sm[];
  __shared__ float s_red[kDThreads / 32];
  if (*d.status & kStatusNoBins) return;
  uint32_t* II = sm;
  // the tiles with container coverage; on the others M_C (1 - O) = 0, dL_u/dO = 0 and the loss
  // partial is 0, as written once per level
  const int n_own = dil_count(d, 0);
  for (int li = blockIdx.x; li < n_own; li += gridDim.x) {
    const int dt = dil_tile(d, 0, li);
    if (!in_bounds(d, dt >= 0 && dt < d.total_dtiles)) continue;
    const int p = find_prob_d(d.prob_dtile_base, d.n_probs, dt);
    const int res = d.prob_res[p], nd = (res + kDT - 1) / kDT, ld = dt - d.prob_dtile_base[p];
    const int x0 = (ld % nd) * kDT, y0 = (ld / nd) * kDT;
    const long long pb = d.prob_pix_base[p];
    const float* Ib = d.img_I + pb;
    const float* Mb = d.covc + pb;
    __syncthreads();
    {  // thread (column, first row): no division per element, 32-bit offsets from the problem's base
      constexpr int CW = DilGeom<K>::CW, RP = kDThreads / CW;
      const int c = threadIdx.x % CW, X = x0 + c - h;
      const bool col_in = X >= 0 && X < res;
      if (c < S) {
#pragma unroll 8
        for (int r = threadIdx.x / CW; r < S; r += RP) {  // unrolled: loads in flight together
          const int Y = y0 + r - h;
          II[(r + 1) * P + c + 1] = col_in && Y >= 0 && Y < res ? to_fixed<K>(1.0f - Ib[Y * res + X]) : 0u;
        }
      }
      if (threadIdx.x < P) II[threadIdx.x] = 0u;              // row 0
      if (threadIdx.x < S) II[(threadIdx.x + 1) * P] = 0u;    // column 0
    }
    // the thread's output item (column c, rows r0..r0 + kVRows - 1): its per-pixel inputs are
    // read now (from a clamped address, used only inside the image), in flight during the scans
    const int c = threadIdx.x % kDT, r0 = (threadIdx.x / kDT) * kVRows;
    const int X = x0 + c, Xc = min(X, res - 1);
    float Iv[kVRows], Mv[kVRows];
#pragma unroll
    for (int i = 0; i < kVRows; ++i) {
      const int o = min(y0 + r0 + i, res - 1) * res + Xc;
      Iv[i] = Ib[o];
      Mv[i] = Mb[o];
    }
    __syncthreads();
    if (threadIdx.x < S) {  // rows: lanes take rows (odd stride, distinct banks)
      uint32_t* row = II + (threadIdx.x + 1) * P + 1;
      uint32_t acc = 0u;
#pragma unroll 9
      for (int c = 0; c < S; ++c) {
        acc += row[c];
        row[c] = acc;
      }
    }
    __syncthreads();
    if (threadIdx.x < S) {  // columns: lanes take columns
      uint32_t* col = II + P + 1 + threadIdx.x;
      uint32_t acc = 0u;
#pragma unroll 9
      for (int r = 0; r < S; ++r) {
        acc += col[r * P];
        col[r * P] = acc;
      }
    }
    __syncthreads();
    float lu = 0.0f;
    {
      // II index of the pixel's own staged position (row r0 + i + h + 1, column c + h + 1)
      const uint32_t* q0 = II + (r0 + h) * P + c + h;
#pragma unroll
      for (int i = 0; i < kVRows; ++i) {
        const int Y = y0 + r0 + i;
        if (X >= res || Y >= res) continue;
        const uint32_t* q = q0 + i * P;
        // s = sum_k w_k (1 - D_k), with 1 - D_k = max(0, 2^Q - B_k) 2^-Q exactly
        float s = 0.0f;
        unsigned mask = 0u;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int r = dil_r(k);
          const uint32_t B = q[(r + 1) * P + r + 1] - q[-r * P + r + 1] - q[(r + 1) * P - r] + q[-r * P - r];
          // B_k may reach 2^32 - 1 (not 2^31): the difference is taken unsigned
          const uint32_t t = (1u << Q) - min(B, 1u << Q);
          if (t != 0u) mask |= 1u << k;  // B_k < 1, decided on the exact fixed-point sum
          s = fmaf(d.L.dil_w[k] * inv_q, (float)t, s);
        }
        const int o = Y * res + X;
        const float O = 1.0f - Iv[i];
        const float M = Mv[i];
        const float mval = M * (1.0f - O);
        lu = fmaf(mval, s, lu);
        d.dil_g[pb + o] = to_fixed<K>(mval) | (mask << 24);  // mval <= 1: at most 2^Q < 2^24
        d.gOu[pb + o] = -(M * s);  // d/dO(q) of M(q)(1 - O(q))(1 - D_k(q)), times M(q)
      }
    }
    // fixed-order block sum
    for (int o = 16; o; o >>= 1) lu += __shfl_xor_sync(0xffffffffu, lu, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = lu;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int i = 0; i < kDThreads / 32; ++i) t += s_red[i];
      d.lossU[dt] = t;
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kDThreads, 6) k_dilate_bwd(Dev d) {
  pdl_enter();
  constexpr int S = DilGeom<K>::S, SP = DilGeom<K>::SP, h = DilGeom<K>::h, Q = DilGeom<K>::Q;
  constexpr float inv_q = 1.0f / (float)(1u << Q);
  extern __shared__ uint32_t sm[];
  if (*d.status & kStatusNoBins) return;
  uint32_t* sM = sm;
  uint32_t* H = sM + S * SP;
  // the tiles with container coverage within the halo (G = 0 over the others and their halos)
  const int n_halo = dil_count(d, 1);
  for (int li = blockIdx.x; li < n_halo; li += gridDim.x) {
    const int dt = dil_tile(d, 1, li);
    if (!in_bounds(d, dt >= 0 && dt < d.total_dtiles)) continue;
    // a tile without coverage of its own was not written by the forward pass: store, not add
    const bool own = (dil_flags(d, dt) & kFlagOwn) != 0;
    const int p = find_prob_d(d.prob_dtile_base, d.n_probs, dt);
    const int res = d.prob_res[p], nd = (res + kDT - 1) / kDT, ld = dt - d.prob_dtile_base[p];
    const int x0 = (ld % nd) * kDT, y0 = (ld / nd) * kDT;
    const long long pb = d.prob_pix_base[p];
    __syncthreads();
    {  // thread (column, first row): no division per element, 32-bit offsets from the problem's base
      constexpr int CW = DilGeom<K>::CW, RP = kDThreads / CW;
      const int c = threadIdx.x % CW, X = x0 + c - h;
      const bool col_in = X >= 0 && X < res;
      const uint32_t* gsrc = d.dil_g + pb;
      if (c < S) {
#pragma unroll 8
        for (int r = threadIdx.x / CW; r < S; r += RP) {  // unrolled: loads in flight together
          const int Y = y0 + r - h;
          const int o = Y * res + X;
          sM[r * SP + c] = col_in && Y >= 0 && Y < res ? gsrc[o] : 0u;
        }
      }
    }
    // the thread's output item (column c, rows r0..r0 + kVRows - 1): the forward pass's direct
    // part of dL_u/dO is read now, in flight during the horizontal pass
    float* g = d.gOu + pb;
    const int c = threadIdx.x % kDT, r0 = (threadIdx.x / kDT) * kVRows;
    const int X = x0 + c, Xc = min(X, res - 1);
    float gv[kVRows];
#pragma unroll
    for (int i = 0; i < kVRows; ++i) gv[i] = own ? g[min(y0 + r0 + i, res - 1) * res + Xc] : 0.0f;
    __syncthreads();
    hsums_all<K>(GSrc{sM, SP}, H);
    __syncthreads();
    float wq[K];
#pragma unroll
    for (int k = 0; k < K; ++k) wq[k] = d.L.dil_w[k] * inv_q;
    {
      uint32_t B[K][kVRows];
      vsums_col<K>(H, c, r0, B);
#pragma unroll
      for (int i = 0; i < kVRows; ++i) {
        const int Y = y0 + r0 + i;
        if (X >= res || Y >= res) continue;
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) acc = fmaf(-wq[k], (float)B[k][i], acc);
        g[Y * res + X] = gv[i] + acc;
      }
    }
  }
}

// Per dilation tile, once per level: whether the container coverage is nonzero on the tile, and
// whether it is nonzero within the halo of the widest kernel; each flag also lists the tile for the
// pass that visits it (the forward pass the first kind, the adjoint the second).
__global__ void k_dtile_flags(Dev d, int h) {
  __shared__ int s_own, s_halo;
  for (int dt = blockIdx.x; dt < d.total_dtiles; dt += gridDim.x) {
    const int p = find_prob_d(d.prob_dtile_base, d.n_probs, dt);
    const int res = d.prob_res[p], nd = (res + kDT - 1) / kDT, ld = dt - d.prob_dtile_base[p];
    const int x0 = (ld % nd) * kDT, y0 = (ld / nd) * kDT;
    const long long pb = d.prob_pix_base[p];
    if (threadIdx.x == 0) s_own = s_halo = 0;
    __syncthreads();
    const int S = kDT + 2 * h;
    int own = 0, halo = 0;
    for (int idx = threadIdx.x; idx < S * S; idx += blockDim.x) {
      const int rr = idx / S, cc = idx % S;
      const int Y = y0 + rr - h, X = x0 + cc - h;
      if (X < 0 || Y < 0 || X >= res || Y >= res) continue;
      if (d.covc[pb + (long long)Y * res + X] > 0.0f) {
        halo = 1;
        if (rr >= h && rr < h + kDT && cc >= h && cc < h + kDT) own = 1;
      }
    }
    if (own) atomicOr(&s_own, 1);
    if (halo) atomicOr(&s_halo, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      d.dtile_flags[dt] = (uint8_t)((s_own ? kFlagOwn : 0) | (s_halo ? kFlagHalo : 0));
      if (s_own) d.dtile_list[atomicAdd(&d.dtile_n[0], 1)] = dt;
      if (s_halo) d.dtile_list[d.total_dtiles + atomicAdd(&d.dtile_n[1], 1)] = dt;
    }
    __syncthreads();
  }
}

// One block per problem: fixed-order float sums of the tile partials (strided per thread, then a
// shuffle tree within and across warps), then Eq. 8.  Float throughout: FP64 arithmetic is slow on
// this part and 1e-7 relative is ample for a sum of non-negative partials.
constexpr int kLossThreads = 1024;
__device__ __forceinline__ float warp_sum_f(float x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__global__ void __launch_bounds__(kLossThreads) k_loss(Dev d) {
  pdl_enter();
  __shared__ float s_red[4][kLossThreads / 32];
  const int p = blockIdx.x;
  const int t0 = d.prob_tile_base[p], t1 = d.prob_tile_base[p + 1];
  const bool use_u = d.L.gamma != 0.0f && d.L.n_dil > 0;
  float a = 0.f, b = 0.f, c = 0.f, u = 0.f;
#pragma unroll 4
  for (int t = t0 + (int)threadIdx.x; t < t1; t += kLossThreads) {
    const float4 v = d.lossA[t];
    a += v.x;
    b += v.y;
    c += v.z;
  }
  if (use_u) {
    const int u0 = d.prob_dtile_base[p], u1 = d.prob_dtile_base[p + 1];
#pragma unroll 4
    for (int t = u0 + (int)threadIdx.x; t < u1; t += kLossThreads) u += d.lossU[t];
  }
  a = warp_sum_f(a);
  b = warp_sum_f(b);
  c = warp_sum_f(c);
  u = warp_sum_f(u);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_red[0][w] = a;
    s_red[1][w] = b;
    s_red[2][w] = c;
    s_red[3][w] = u;
  }
  __syncthreads();
  if (w == 0) {
    a = warp_sum_f(s_red[0][lane]);
    b = warp_sum_f(s_red[1][lane]);
    c = warp_sum_f(s_red[2][lane]);
    u = warp_sum_f(s_red[3][lane]);
    if (lane == 0) {
      const float np = (float)d.prob_res[p] * (float)d.prob_res[p];
      const float Lc = a / np, Lo = b / np, Ld = c / np;
      float* out = d.loss_terms + 5 * p;
      out[0] = Lc;
      out[1] = Lo;
      out[2] = u;
      out[3] = Ld;
      out[4] = d.L.alpha * Lc + d.L.beta * Lo + d.L.gamma * u + d.L.delta * Ld;
    }
  }
}

// Deterministic mode: each element sums its (tile, element) partials over its tile rectangle, one
// warp per element: lane l takes the tiles l, l + 32, ... of the rectangle in row-major order (a
// tile's list is ordered by element id, so the pair is found by bisection) and the 32 lane sums are
// added by a fixed shuffle tree; the order of every addition is fixed, so the result is bitwise
// reproducible.
constexpr int kReduceWarps = 8;
__global__ void __launch_bounds__(kReduceWarps * 32) k_grad_reduce(Dev d, int mark) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int g = blockIdx.x * kReduceWarps + (threadIdx.x >> 5);
  if (g < d.n_elems && !(*d.status & kStatusNoBins)) {
    const int4 rc = d.rect[g];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (rc.z >= rc.x && rc.w >= rc.y) {
      const int p = d.elem_prob[g];
      const int tb = d.prob_tile_base[p], ntx = d.prob_ntx[p];
      const int w = rc.z - rc.x + 1, n = w * (rc.w - rc.y + 1);
      for (int i = lane; i < n; i += 32) {
        const int t = tb + (rc.y + i / w) * ntx + rc.x + i % w;
        const int* sorted = d.tile_sorted + (size_t)t * d.tile_cap;
        const int m = d.tile_m[t];
        int lo = 0, hi = m;  // first entry >= g
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (sorted[mid] < g) lo = mid + 1;
          else hi = mid;
        }
        const int sl = lo < m ? d.tile_sorted_slot[(size_t)t * d.tile_cap + lo] : -1;
        if (lo < m && sorted[lo] == g && in_bounds(d, sl >= 0 && sl < d.cap)) {
          const float4 v = d.partial[sl];
          acc.x += v.x;
          acc.y += v.y;
          acc.z += v.z;
          acc.w += v.w;
        }
      }
    }
    for (int o = 16; o; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
      acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    }
    if (lane == 0) d.dq[g] = acc;
  }
  if (mark) mark_step_if_last(d);
}

// Applies a pending Adam step to every element (see adam_update); the last block to finish clears
// the flag, once every block has read it.  With `out`, also gathers the params, the loss terms and
// the control words (status, step, pair count, 0) into one buffer, [4n | 5 n_probs | 4], so that one
// copy brings all of them to the host.
__global__ void k_adam_flush(Dev d, float* out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const bool pend = *d.pending != 0;
  if (g < d.n_elems) {
    if (pend && !d.fit) adam_update(d, g, *d.step, d.dq[g]);
    if (out) reinterpret_cast<float4*>(out)[g] = d.q[g];
  }
  if (out && blockIdx.x == 0) {
    float* tail = out + 4 * (size_t)d.n_elems;
    for (int i = threadIdx.x; i < 5 * d.n_probs; i += blockDim.x) tail[i] = d.loss_terms[i];
    if (threadIdx.x == 0) {
      int* c = reinterpret_cast<int*>(tail + 5 * d.n_probs);
      for (int i = 0; i < kCtlWords; ++i) c[i] = d.status[i];  // the control words, in order
      c[3] = 0;  // the pending step is applied by this flush
    }
  }
  __syncthreads();  // every thread of the block has read the flag
  if (threadIdx.x == 0 && atomicAdd(&d.work[5], 1) == (int)gridDim.x - 1) {
    *d.pending = 0;
    d.work[5] = 0;
  }
}

static size_t dilate_smem(int K, bool backward) {
  const int S = kDT + 2 * dil_r(K - 1), SP = S | 1;
  // the forward pass keeps one integral image with a zero row and column; the backward pass stages
  // the packed words the forward pass wrote and keeps every kernel's horizontal sums
  if (!backward) return (size_t)(S + 1) * (S + 1) * sizeof(uint32_t);
  const size_t f = (size_t)S * SP + (size_t)hbase(K) * kHP;
  return f * sizeof(uint32_t);
}

template <int K>
static cudaError_t prepare_k() {
  cudaError_t e = cudaFuncSetAttribute(k_dilate_bwd<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)dilate_smem(K, true));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_dilate_fwd<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)dilate_smem(K, false));
}

cudaError_t prepare_dilate(int n_dil) {
  switch (n_dil) {
    case 1: return prepare_k<1>();
    case 2: return prepare_k<2>();
    case 3: return prepare_k<3>();
    case 4: return prepare_k<4>();
    case 5: return prepare_k<5>();
    case 6: return prepare_k<6>();
    case 7: return prepare_k<7>();
    case 8: {  // the largest: also raise every smaller instantiation (callers may mix sizes)
      for (int k = 1; k < 8; ++k) {
        cudaError_t e = prepare_dilate(k);
        if (e != cudaSuccess) return e;
      }
      return prepare_k<8>();
    }
    default: return cudaSuccess;
  }
}

template <int K>
static cudaError_t launch_k(const Dev& d, cudaStream_t s, bool backward) {
  const size_t sm = dilate_smem(K, backward);
  if (backward) return klaunch(d.pdl, k_dilate_bwd<K>, d.total_dtiles, kDThreads, sm, s, d);
  return klaunch(d.pdl, k_dilate_fwd<K>, d.total_dtiles, kDThreads, sm, s, d);
}

cudaError_t launch_dilate(const Dev& d, cudaStream_t s, bool backward) {
  switch (d.L.n_dil) {
    case 1: return launch_k<1>(d, s, backward);
    case 2: return launch_k<2>(d, s, backward);
    case 3: return launch_k<3>(d, s, backward);
    case 4: return launch_k<4>(d, s, backward);
    case 5: return launch_k<5>(d, s, backward);
    case 6: return launch_k<6>(d, s, backward);
    case 7: return launch_k<7>(d, s, backward);
    case 8: return launch_k<8>(d, s, backward);
    default: return cudaSuccess;
  }
}

cudaError_t launch_dtile_flags(const Dev& d, cudaStream_t s) {
  if (d.L.n_dil <= 0 || !d.dtile_flags || !d.dtile_list) return cudaSuccess;
  k_dtile_flags<<<d.total_dtiles, 256, 0, s>>>(d, dil_r(d.L.n_dil - 1));
  return cudaGetLastError();
}

cudaError_t launch_loss(const Dev& d, cudaStream_t s) {
  return klaunch(d.pdl, k_loss, d.n_probs, kLossThreads, 0, s, d);
}

cudaError_t launch_grad_reduce(const Dev& d, cudaStream_t s, bool mark_step) {
  return klaunch(d.pdl, k_grad_reduce, (d.n_elems + kReduceWarps - 1) / kReduceWarps, kReduceWarps * 32, 0,
                 s, d, mark_step ? 1 : 0);
}

cudaError_t launch_adam_flush(const Dev& d, cudaStream_t s, float* out) {
  k_adam_flush<<<(d.n_elems + 255) / 256, 256, 0, s>>>(d, out);
  return cudaGetLastError();
}

cudaError_t launch_copy_grad(const Dev& d, cudaStream_t s, float* out) {
  return cudaMemcpyAsync(out, d.dq, sizeof(float4) * (size_t)d.n_elems, cudaMemcpyDeviceToDevice, s);
}

}  // namespace collage
