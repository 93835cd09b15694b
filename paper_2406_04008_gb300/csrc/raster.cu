// Tile rasteriser (forward), its adjoint, and the container raster.
//
// Coverage of element i at pixel p is c = S(sd / rho) with sd the signed distance (winding number
// for the sign, positive inside; hw - d for open strokes) and S(x) = (1 + x)^2 (2 - x) / 4 on
// [-1, 1] (the same cubic as 1/2 + 3x/4 - x^3/4, written in factored form so that 1 - S(x) =
// S(-x) keeps full relative precision near x = 1).  This is the anti-aliased, differentiable
// rasteriser the method builds on (Sec. 3 "Differentiable Rendering"); the composites and
// per-pixel losses are those of Sec. 4.2 (Eqs. 5, 6 and the force term of Sec. 5).
//
// Precision: each element's vertices are stored relative to its translation, in pixels, and the
// pixel is brought into that frame as (p - t_hi) - t_lo, so every FP32 quantity is a few tens of
// pixels at most and the signed distance carries an error of ~1e-6 px at any grid size.
//
// The forward pass saves, for every (tile, element) pair and pixel of the tile, the signed
// distance and the closest segment; the adjoint reads them back instead of repeating the segment
// loop, so only one pass over the pixel-segment pairs happens per iteration.  Pixels farther than
// the coverage margin from the outline carry sd = +-1e30 (saturated coverage, no gradient).
#include <cfloat>

#include "internal.h"

namespace collage {

__device__ __forceinline__ float Sfun(float x) {
  x = fminf(fmaxf(x, -1.0f), 1.0f);
  const float a = 1.0f + x;
  return 0.25f * a * a * (2.0f - x);
}
__device__ __forceinline__ float dSfun(float x) {
  x = fminf(fmaxf(x, -1.0f), 1.0f);
  return 0.75f * (1.0f - x) * (1.0f + x);
}

__device__ __forceinline__ int find_prob(const int* base, int P, int tile) {
  int lo = 0, hi = P - 1;  // last p with base[p] <= tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Distance / winding update of one point against one staged segment (a, a + e) whose end point
// has y = b_y.  Winding: the segment crosses the +x ray from the point when the two end points lie
// on different sides of it (half-open in y); cross(e, w) > 0 puts the crossing right of the point
// for an upward segment, < 0 for a downward one.
struct SegQuery {
  float best;  // squared distance
  int idx;
  int wn;
};

__device__ __forceinline__ void seg_update(SegQuery& Q, float dx, float dy, float4 s, float2 s2,
                                           int j, bool winding) {
  const float wx = dx - s.x, wy = dy - s.y;
  const float t = __saturatef((wx * s.z + wy * s.w) * s2.y);
  const float qx = fmaf(-t, s.z, wx), qy = fmaf(-t, s.w, wy);
  const float d2 = fmaf(qx, qx, qy * qy);
  if (d2 < Q.best) {
    Q.best = d2;
    Q.idx = j;
  }
  if (winding) {
    const bool a_le = wy >= 0.0f;         // a.y <= p.y
    const bool b_le = dy - s2.x >= 0.0f;  // b.y <= p.y
    const float cr = s.z * wy - s.w * wx;
    if (a_le && !b_le && cr > 0.0f) Q.wn += 1;
    if (!a_le && b_le && cr < 0.0f) Q.wn -= 1;
  }
}

constexpr int kSegCap = 1024;   // container segments staged per chunk
constexpr int kNearCap = 64;    // near segments staged per chunk of one (tile, element) pair
constexpr int kRowCross = 16;   // crossings listed per pixel row of a pair
constexpr int kPairWarps = 4;   // pairs per block of the per-pair adjoint (one per warp)
constexpr float kFar = 1e30f;   // |sd| of a pixel farther than the coverage margin

__device__ __forceinline__ void tile_coords(const Dev& d, int tile, int T, int& p, int& tx, int& ty,
                                            int& res) {
  p = find_prob(d.prob_tile_base, d.n_probs, tile);
  const int lt = tile - d.prob_tile_base[p], ntx = d.prob_ntx[p];
  res = d.prob_res[p];
  tx = lt % ntx;
  ty = lt / ntx;
}

// ------------------------------------------------------------------------------------------------
// Signed distances of one near (tile, element) pair per block (the emission lists the near pairs;
// the others have saturated coverage on the whole tile and need no per-pixel work).
//
// The block first splits the outline's segments.  A segment whose box meets the tile's pixel-centre
// box grown by the coverage margin m = rho + pad (+ stroke half-width) is "near": warp 0 appends
// it, in index order, to a shared list.  Every other segment lies farther than m from every pixel
// of the tile; if it spans a pixel row and lies right of the grown box it crosses that row's +x
// ray right of every pixel, so the other warps add its +-1 to a per-row winding backdrop.  A pixel
// then runs the distance and crossing tests over the near list only: its winding is backdrop +
// near crossings; if no near segment is within m the coverage is saturated (0 or 1, as the full
// loop would give) and sd = +-1e30, else the near minimum is the true distance.
// ------------------------------------------------------------------------------------------------
// Winding number of a point (element frame) over every segment of an outline: the crossing test of
// the distance kernel applied to all segments (the far ones are well conditioned).
__device__ __noinline__ int winding_all(const Dev& d, int v0, int ns, float px, float py) {
  int w = 0;
  for (int j = 0; j < ns; ++j) {
    const float4 sa = d.segA[v0 + j];
    const float wy = py - sa.y;
    const bool a_le = wy >= 0.0f, b_le = py - d.segB[v0 + j].x >= 0.0f;
    if (a_le != b_le && px < fmaf(wy, d.segS[v0 + j], sa.x)) w += a_le ? 1 : -1;
  }
  return w;
}

template <int T, int NT>
__global__ void __launch_bounds__(NT, NT == 64 ? 16 : 1024 / NT) k_pair_sd(Dev d) {
  pdl_enter();
  constexpr int NP = T * T, PPT = NP / NT, NW = NT / 32;
  static_assert(NW >= 2, "warp 0 compacts near segments, the others count the winding backdrop");
  __shared__ float4 s_seg[kNearCap];
  __shared__ float2 s_seg2[kNearCap];
  __shared__ float s_slope[kNearCap];
  __shared__ int s_idx[kNearCap];
  __shared__ int s_back[T];
  __shared__ float s_rx[T][kRowCross];  // per pixel row: x of its crossings with near segments
  __shared__ signed char s_rd[T][kRowCross];  // and their direction
  __shared__ int s_rc[T];
  __shared__ int s_near;
  if (*d.status & kStatusOverflow) return;
  const float inv_rho = 1.0f / d.L.rho_px, pad = d.L.pad_px;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n_heavy = d.work[2], n_near = n_heavy + d.work[4];
  // the near pairs: a block's first is its block index in the list, the others are taken from a
  // shared counter as blocks finish (pair costs vary by two orders of magnitude); s_next is
  // double-buffered so that thread 0's next write never meets a read of the previous value
  __shared__ int s_next[2];
  constexpr int kLiveBatch = 8;
  __shared__ int4 s_live[kLiveBatch];
  int n_live = 0;  // thread 0's count of buffered live records
  for (int i = blockIdx.x, it = 0; i < n_near; ++it) {
    if (threadIdx.x == 0) s_next[it & 1] = (int)gridDim.x + atomicAdd(&d.work[0], 1);
    const int4 rec = d.near_list[i < n_heavy ? i : d.cap - 1 - (i - n_heavy)];
    const int slot = rec.x, g = rec.y, txy = rec.z;
    const int tx = txy & 0xffff, ty = txy >> 16, p = rec.w, res = d.prob_res[p];
    const int v0 = d.elem_voff[g], nv = d.elem_voff[g + 1] - v0;
    const bool closed = d.elem_closed[g] != 0;
    const int ns = closed ? nv : nv - 1;
    const float4 tp = d.tpx[g], bb = d.bbox[g];
    const float hwpx = closed ? 0.0f : d.elem_hw[g] * (float)res;
    const float mrg = d.L.rho_px + pad + hwpx;
    const float mrg2 = mrg * mrg;
    // tile pixel-centre box in the element frame, grown by the margin (+ rounding slack)
    const float cx0 = (float)(tx * T) + 0.5f, cx1 = (float)(tx * T + T) - 0.5f;
    const float cy0 = (float)(ty * T) + 0.5f, cy1 = (float)(ty * T + T) - 0.5f;
    const float gx0 = (cx0 - tp.x) - tp.z - mrg - 0.01f, gx1 = (cx1 - tp.x) - tp.z + mrg + 0.01f;
    const float gy0 = (cy0 - tp.y) - tp.w - mrg - 0.01f, gy1 = (cy1 - tp.y) - tp.w + mrg + 0.01f;
    float dx[PPT], dy[PPT], best[PPT];
    int bj[PPT], wn[PPT], idx[PPT];
    bool act[PPT];
    bool any = false;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int local = threadIdx.x + k * NT;
      const int X = tx * T + local % T, Y = ty * T + local / T;
      dx[k] = ((float)X + 0.5f - tp.x) - tp.z;
      dy[k] = ((float)Y + 0.5f - tp.y) - tp.w;
      act[k] = X < res && Y < res && dx[k] >= bb.x && dx[k] <= bb.z && dy[k] >= bb.y && dy[k] <= bb.w;
      any |= act[k];
      best[k] = FLT_MAX;
      idx[k] = 0;
      bj[k] = -1;
      wn[k] = 0;
    }
    // the compaction (warp 0) and the backdrop (the other warps) read the outline from global
    // memory side by side: the second reader finds it in L1, and no block-wide staging round and
    // barrier precede them
    const float4* SA = d.segA + v0;
    const float2* SB = d.segB + v0;
    const float* SS = d.segS + v0;
    for (int base = 0;; base += kNearCap) {
      __syncthreads();  // the previous users of the shared lists are done
      if (wid == 0) {
        // ordered compaction of the near segments with positions in [base, base + kNearCap)
        int cnt = 0;
        for (int j0 = 0; j0 < ns; j0 += 32) {
          const int j = j0 + lane;
          bool nr = false;
          float4 sa = make_float4(0.f, 0.f, 0.f, 0.f);
          float2 sb = make_float2(0.f, 0.f);
          if (j < ns) {
            sa = SA[j];
            sb = SB[j];
            const float bx = sa.x + sa.z;
            nr = !(fmaxf(sa.x, bx) < gx0 || fminf(sa.x, bx) > gx1 || fmaxf(sa.y, sb.x) < gy0 ||
                   fminf(sa.y, sb.x) > gy1);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, nr);
          const int pos = cnt + __popc(bal & ((1u << lane) - 1u)) - base;
          if (nr && pos >= 0 && pos < kNearCap) {
            s_seg[pos] = sa;
            s_seg2[pos] = sb;
            s_slope[pos] = SS[j];
            s_idx[pos] = j;
          }
          cnt += __popc(bal);
        }
        if (lane == 0) s_near = cnt;
      } else if (base == 0 && closed) {
        // winding backdrop of the far segments right of the tile
        for (int r = threadIdx.x - 32; r < T; r += NT - 32) {
          s_back[r] = 0;
          s_rc[r] = 0;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(NT - 32));
        // the rows' dy as the pixels form them: non-decreasing in the row, so a segment whose y
        // range misses [first row, last row] crosses no row's ray
        const float yr0 = ((float)(ty * T) + 0.5f - tp.y) - tp.w;
        const float yr1 = ((float)(ty * T + T - 1) + 0.5f - tp.y) - tp.w;
        for (int j = threadIdx.x - 32; j < ns; j += NT - 32) {
          const float4 sa = SA[j];
          const float2 sb = SB[j];
          if (fminf(sa.x, sa.x + sa.z) <= gx1) continue;  // near, left or overlapping in x
          if (fmaxf(sa.y, sb.x) <= yr0 || fminf(sa.y, sb.x) > yr1) continue;
          const int up = sa.y < sb.x ? 1 : -1;
          for (int r = 0; r < T; ++r) {
            const float yr = ((float)(ty * T + r) + 0.5f - tp.y) - tp.w;  // as a pixel forms dy
            if ((yr >= sa.y) != (yr >= sb.x)) atomicAdd(&s_back[r], up);
          }
        }
      }
      __syncthreads();
      const int total_near = s_near;
      const int cn = min(kNearCap, total_near - base);
      if (closed && cn > 0) {
        // the crossings of the pixel rows with the chunk's near segments, listed per row.  Row r
        // crosses segment j when its end points lie on different sides of the row (half-open, on
        // the dy the pixels form); the crossing counts for a pixel left of its x, +1 upward and
        // -1 downward.  (x of the crossing instead of the sign of cross(e, p - a): the two differ
        // only for a pixel within rounding of the segment, where sd ~ 0 and c ~ 1/2 either way.)
        for (int e = threadIdx.x; e < cn * T; e += NT) {
          const int j = e / T, r = e % T;
          const float4 sa = s_seg[j];
          const float yr = ((float)(ty * T + r) + 0.5f - tp.y) - tp.w;
          const bool a_le = yr - sa.y >= 0.0f, b_le = yr - s_seg2[j].x >= 0.0f;
          if (a_le != b_le) {
            const int q = atomicAdd(&s_rc[r], 1);
            if (q < kRowCross) {
              s_rx[r][q] = fmaf(yr - sa.y, s_slope[j], sa.x);
              s_rd[r][q] = a_le ? 1 : -1;
            }
          }
        }
      }
      if (any && cn > 0) {
#pragma unroll 2
        for (int j = 0; j < cn; ++j) {
          const float4 s = s_seg[j];
          const float ie = s_seg2[j].y;
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            if (!act[k]) continue;
            const float wx = dx[k] - s.x, wy = dy[k] - s.y;
            const float t = __saturatef((wx * s.z + wy * s.w) * ie);
            const float qx = fmaf(-t, s.z, wx), qy = fmaf(-t, s.w, wy);
            const float d2 = fmaf(qx, qx, qy * qy);
            if (d2 < best[k]) {
              best[k] = d2;
              bj[k] = j;
            }
          }
        }
#pragma unroll
        for (int k = 0; k < PPT; ++k)  // a minimum set in this chunk: its segment index
          if (bj[k] >= 0) {
            idx[k] = s_idx[bj[k]];
            bj[k] = -1;
          }
      }
      if (total_near <= base + kNearCap) break;
    }
    if (closed) __syncthreads();  // the row crossing lists are complete
    if (d.paths) {
      if (closed && threadIdx.x < T && s_rc[threadIdx.x] > kRowCross) atomicAdd(&d.paths[0], 1ull);
      if (threadIdx.x == 0 && s_near > kNearCap) atomicAdd(&d.paths[1], 1ull);
    }
    float2* sv = d.saved + (size_t)slot * NP;
    bool live = false;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      float sd = -kFar;
      if (act[k] && closed) {
        const int row = (threadIdx.x + k * NT) / T, rc = s_rc[row];
        if (rc <= kRowCross) {
          wn[k] = s_back[row];
          for (int q = 0; q < rc; ++q)
            if (dx[k] < s_rx[row][q]) wn[k] += s_rd[row][q];
        } else {  // a row crossing the outline more often than the list holds: all segments
          wn[k] = winding_all(d, v0, ns, dx[k], dy[k]);
        }
      }
      if (act[k]) {
        const int w = closed ? wn[k] : 0;
        if (best[k] < mrg2) {
          const float dist = sqrtf(best[k]);
          sd = closed ? (w != 0 ? dist : -dist) : hwpx - dist;
        } else {
          sd = (closed && w != 0) ? kFar : -kFar;
        }
        live |= fabsf(sd * inv_rho) < 1.0f || fabsf((sd + pad) * inv_rho) < 1.0f;
      }
      sv[threadIdx.x + k * NT] = make_float2(sd, __int_as_float(idx[k]));
    }
    live = __syncthreads_or(live);
    if (threadIdx.x == 0) {
      if (live) {
        // live pairs are appended kLiveBatch at a time: one atomic per batch
        s_live[n_live++] = rec;
        if (n_live == kLiveBatch) {
          const int at = atomicAdd(&d.work[1], kLiveBatch);
          for (int q = 0; q < kLiveBatch; ++q) d.live_list[at + q] = s_live[q];
          n_live = 0;
        }
      } else if (d.deterministic) {
        d.partial[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    i = s_next[it & 1];
  }
  if (threadIdx.x == 0 && n_live > 0) {
    const int at = atomicAdd(&d.work[1], n_live);
    for (int q = 0; q < n_live; ++q) d.live_list[at + q] = s_live[q];
  }
}

// ------------------------------------------------------------------------------------------------
// Composite, one tile per warp: order the tile's pairs by element id (ids are unique in a tile, so
// an id's rank is the number of smaller ids; for up to 32 pairs the lanes hold the ids and rank
// them by shuffles), then per pixel Ihat = prod(1 - c_i) and prod(1 - tau c_i^pad) over the pairs
// in that order, and the per-pixel loss terms (Eq. 5, Eq. 6 surrogate, force), summed over the
// tile by a fixed shuffle tree.  No block-wide barrier: each warp owns its tile.
// ------------------------------------------------------------------------------------------------
constexpr int kCompWarps = 4;
template <int T>
__global__ void __launch_bounds__(kCompWarps * 32) k_composite(Dev d, float* out_bw, float* out_tau) {
  pdl_enter();
  constexpr int NP = T * T, PPL = NP / 32;
  __shared__ int s_slot[kCompWarps][32];
  __shared__ uint8_t s_cls[kCompWarps][32];
  if (*d.status & kStatusOverflow) return;
  const float inv_rho = 1.0f / d.L.rho_px, pad = d.L.pad_px, tau = d.L.tau;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int* w_slot = s_slot[wid];
  uint8_t* w_cls = s_cls[wid];
  for (int tile = blockIdx.x * kCompWarps + wid; tile < d.total_tiles; tile += gridDim.x * kCompWarps) {
    int p, tx, ty, res;
    tile_coords(d, tile, T, p, tx, ty, res);
    const long long pixbase = d.prob_pix_base[p];
    const uint2 rg = d.range[tile];
    const int m = (int)(rg.y - rg.x);
    const bool small = m <= 32;
    __syncwarp();  // the previous tile's readers of this warp's lists are done
    if (small) {
      const int v = lane < m ? d.pair_elem[rg.x + lane] : 0;
      int r = 0;
      for (int j = 0; j < m; ++j) r += __shfl_sync(0xffffffffu, v, j) < v ? 1 : 0;
      if (lane < m) {
        w_slot[r] = (int)rg.x + lane;
        w_cls[r] = d.pair_cls[rg.x + lane];
        d.pair_sorted[rg.x + r] = v;
        d.pair_slot[rg.x + r] = (int)rg.x + lane;
      }
    } else {
      if (lane == 0 && d.paths) atomicAdd(&d.paths[2], 1ull);
      for (int i = lane; i < m; i += 32) {
        const int vi = d.pair_elem[rg.x + i];
        int r = 0;
        for (int j = 0; j < m; ++j) r += d.pair_elem[rg.x + j] < vi ? 1 : 0;
        d.pair_sorted[rg.x + r] = vi;
        d.pair_slot[rg.x + r] = (int)rg.x + i;
      }
    }
    __syncwarp();  // the ordered list is visible to the whole warp
    // products over the pairs in element order; the pair loop is outermost so that a lane's loads
    // of its PPL pixels are independent and in flight together
    float keep[PPL], keept[PPL];
    int zc[PPL], nfull[PPL];
    bool partial[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      keep[k] = 1.0f;
      keept[k] = 1.0f;
      zc[k] = 0;
      nfull[k] = 0;
      partial[k] = false;
    }
    for (int i = 0; i < m; ++i) {
      const int slot = small ? w_slot[i] : d.pair_slot[rg.x + i];
      const uint8_t cls = small ? w_cls[i] : d.pair_cls[slot];
      if (cls == kPairOut) continue;  // c = c^pad = 0: factors of 1
      float sd[PPL];
#pragma unroll
      for (int k = 0; k < PPL; ++k)  // an inside pair has c = c^pad = 1: sd = +1e30 gives that
        sd[k] = cls == kPairIn ? kFar : d.saved[(size_t)slot * NP + lane + 32 * k].x;
#pragma unroll
      for (int k = 0; k < PPL; ++k) {
        const float x = sd[k] * inv_rho;
        const float omc = Sfun(-x), cp = Sfun((sd[k] + pad) * inv_rho);
        if (omc == 0.0f) zc[k] += 1;
        else keep[k] *= omc;
        keept[k] *= 1.0f - tau * cp;
        nfull[k] += cp == 1.0f;
        partial[k] |= cp > 0.0f && cp < 1.0f;
      }
    }
    float lc = 0.0f, lo = 0.0f, ld = 0.0f;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int local = lane + 32 * k;
      const int X = tx * T + local % T, Y = ty * T + local / T;
      if (X >= res || Y >= res) continue;
      const long long pix = pixbase + (long long)Y * res + X;
      const float ihat = zc[k] ? 0.0f : keep[k];
      const float cov = d.covc[pix];
      const float W = cov >= 0.5f ? d.L.w_in : d.L.w_out;
      const float df = ihat - (1.0f - cov);
      lc += W * df * df;
      const float A = 1.0f - keept[k];
      // the kink of max(0, A - tau): one fully covering element gives A = tau exactly and any
      // other element with c^pad > 0 lifts A above it, by less than float can resolve when that
      // c^pad is tiny; so the side of the kink is taken from the counts in that case (exact)
      const bool over = nfull[k] >= 2 || (nfull[k] == 1 ? partial[k] : A > tau);
      lo += over ? fmaxf(A - tau, 0.0f) : 0.0f;
      ld += (1.0f - ihat) * force_potential(d.L, ((float)X + 0.5f) / (float)res, ((float)Y + 0.5f) / (float)res);
      d.img_I[pix] = ihat;
      d.img_Pt[pix] = over ? -keept[k] : keept[k];  // the sign carries the side of the kink
      if (out_bw) out_bw[pix] = ihat;
      if (out_tau) out_tau[pix] = A;
    }
    for (int o = 16; o; o >>= 1) {  // fixed-order sums of the three partials
      lc += __shfl_xor_sync(0xffffffffu, lc, o);
      lo += __shfl_xor_sync(0xffffffffu, lo, o);
      ld += __shfl_xor_sync(0xffffffffu, ld, o);
    }
    if (lane == 0) d.lossA[tile] = make_float4(lc, lo, ld, 0.0f);
  }
}

// ------------------------------------------------------------------------------------------------
// Adjoint, one (tile, element) pair per warp: dL/dIhat and dL/dA_tau per pixel, then the chain
// dL/dc -> dc/dsd -> dsd/d(closest segment) -> d/d(tx, ty, theta, s) of Eq. 2, reduced over the
// tile's pixels by a fixed shuffle tree and added to the element's gradient (or stored per pair).
// ------------------------------------------------------------------------------------------------
template <int T, bool FIT>  // FIT: also dL/d(vertex) for outline fitting (d.fit)
__global__ void __launch_bounds__(kPairWarps * 32) k_raster_bwd(Dev d, int mark) {
  pdl_enter();
  constexpr int NP = T * T, PPL = NP / 32;
  if (*d.status & kStatusOverflow) return;
  const float inv_rho = 1.0f / d.L.rho_px, pad = d.L.pad_px, tau = d.L.tau;
  const bool use_u = d.L.gamma != 0.0f;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n_live = d.work[1];  // pairs without a gradient-carrying pixel are not listed
  const int stride = (int)gridDim.x * kPairWarps;
  int i = blockIdx.x * kPairWarps + wid;
  int4 rec = i < n_live ? d.live_list[i] : make_int4(0, 0, 0, 0);
  for (; i < n_live; i += stride) {
    // the next pair's record is read while this one is worked on
    const int4 rec_next = i + stride < n_live ? d.live_list[i + stride] : rec;
    const int slot = rec.x, g = rec.y, txy = rec.z, p = rec.w;
    const int tx = txy & 0xffff, ty = txy >> 16, res = d.prob_res[p];
    const long long pixbase = d.prob_pix_base[p];
    const float inv_np = 1.0f / ((float)res * (float)res);
    const int v0 = d.elem_voff[g];
    const bool closed = d.elem_closed[g] != 0;
    const float4 tp = d.tpx[g];
    const float4 qg = d.q[g];
    const float s_inv = 1.0f / qg.w;
    const float2* sv = d.saved + (size_t)slot * NP;
    // outline fitting: d(pixel)/d(local vertex) = s res R(theta), applied transposed below
    float fc = 0.0f, fs = 0.0f, sres = 0.0f;
    int nv = 0;
    if (FIT) {
      sincosf(qg.z, &fs, &fc);
      sres = qg.w * (float)res;
      nv = d.elem_voff[g + 1] - v0;
    }
    // every per-pixel input of the warp's pixels in one round of loads
    float2 srec[PPL];
    float ihat[PPL], pt_s[PPL], cov[PPL], gou[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int local = lane + 32 * k;
      const int X = tx * T + local % T, Y = ty * T + local / T;
      srec[k] = make_float2(kFar, 0.0f);
      ihat[k] = pt_s[k] = cov[k] = gou[k] = 0.0f;
      if (X < res && Y < res) {
        const long long pix = pixbase + (long long)Y * res + X;
        srec[k] = sv[local];
        ihat[k] = d.img_I[pix];
        pt_s[k] = d.img_Pt[pix];
        cov[k] = d.covc[pix];
        if (use_u) gou[k] = d.gOu[pix];
      }
    }
    // dL/dsd per pixel, then the closest segments of the pixels that carry a gradient
    float gsd[PPL];
    float4 sa[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int local = lane + 32 * k;
      const int X = tx * T + local % T, Y = ty * T + local / T;
      const float sd = srec[k].x;
      const float x = sd * inv_rho, xp = (sd + pad) * inv_rho;
      gsd[k] = 0.0f;
      if (fabsf(x) < 1.0f || fabsf(xp) < 1.0f) {  // never for the out-of-range pixels (sd = 1e30)
        const float pt = fabsf(pt_s[k]);  // negative: the pixel is on the rising side of the Eq. 6 kink
        const float W = cov[k] >= 0.5f ? d.L.w_in : d.L.w_out;
        const float py = (float)Y + 0.5f;
        // O = 1 - Ihat: the uniform and force terms enter dL/dIhat with a minus sign
        const float gI = d.L.alpha * inv_np * 2.0f * W * (ihat[k] - (1.0f - cov[k])) - d.L.gamma * gou[k] -
                         d.L.delta * inv_np *
                             force_potential(d.L, ((float)X + 0.5f) / (float)res, py / (float)res);
        const float gA = pt_s[k] < 0.0f ? d.L.beta * inv_np : 0.0f;
        const float omc = Sfun(-x), cp = Sfun(xp);
        // dIhat/dc_i = -prod_{j != i}(1 - c_j) = -Ihat / (1 - c_i)   (0 when another c_j = 1)
        const float gc = omc > 0.0f ? -gI * ihat[k] / omc : 0.0f;
        // dA/dc^pad_i = tau prod_{j != i}(1 - tau c^pad_j)
        const float gcp = gA * tau * pt / (1.0f - tau * cp);
        gsd[k] = (gc * dSfun(x) + gcp * dSfun(xp)) * inv_rho;
      }
      if (gsd[k] != 0.0f) sa[k] = d.segA[v0 + __float_as_int(srec[k].y)];
    }
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      if (gsd[k] == 0.0f) continue;
      const int local = lane + 32 * k;
      const int X = tx * T + local % T, Y = ty * T + local / T;
      const float sd = srec[k].x;
      const float dx = ((float)X + 0.5f - tp.x) - tp.z, dy = ((float)Y + 0.5f - tp.y) - tp.w;
      const float ex = sa[k].z, ey = sa[k].w, ee = ex * ex + ey * ey;
      const float wx = dx - sa[k].x, wy = dy - sa[k].y;
      const float u = ee > 0.0f ? __saturatef((wx * ex + wy * ey) / ee) : 0.0f;
      const float qx = fmaf(u, ex, sa[k].x), qy = fmaf(u, ey, sa[k].y);  // closest point, rel. to t
      // unit normal from the closest point towards the pixel: for a closest point inside the
      // segment it is the segment's perpendicular on the pixel's side (well conditioned even
      // when the pixel is almost on the outline); at an end point it is the direction to the pixel
      float nx, ny;
      if (u > 0.0f && u < 1.0f) {
        const float inv_len = rsqrtf(ee);
        const float side = ex * wy - ey * wx >= 0.0f ? inv_len : -inv_len;
        nx = -ey * side;
        ny = ex * side;
      } else {
        const float rx = dx - qx, ry = dy - qy;
        const float dist = sqrtf(rx * rx + ry * ry);
        if (!(dist > 0.0f)) continue;
        nx = rx / dist;
        ny = ry / dist;
      }
      // sd = sig * dist (closed: sig = +-1 by the winding; open: sd = hw - dist, sig = -1)
      const float sig = closed ? (sd > 0.0f ? 1.0f : -1.0f) : -1.0f;
      const float gs = -sig * gsd[k];
      a0 += gs * nx * (float)res;              // d(dist)/dt = -n, t in unit coords
      a1 += gs * ny * (float)res;
      a2 += gs * (ny * qx - nx * qy);          // d(dist)/dtheta = -n . J q
      a3 += gs * (nx * qx + ny * qy) * s_inv;  // d(dist)/ds = -n . q / s
      if (FIT) {
        // d(dist)/d(end points) = -n (1 - u), -n u (the closest point moves with them), taken to
        // element-local unit coordinates
        const float gx = gs * nx, gy = gs * ny;
        const float lx = sres * (fc * gx + fs * gy), ly = sres * (fc * gy - fs * gx);
        const int j = __float_as_int(srec[k].y);
        const int ja = v0 + j, jb = v0 + (j + 1 == nv ? 0 : j + 1);
        atomicAdd(&d.dv[ja].x, lx * (1.0f - u));
        atomicAdd(&d.dv[ja].y, ly * (1.0f - u));
        atomicAdd(&d.dv[jb].x, lx * u);
        atomicAdd(&d.dv[jb].y, ly * u);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
      a3 += __shfl_xor_sync(0xffffffffu, a3, o);
    }
    if (lane == 0) {
      if (d.deterministic) {
        d.partial[slot] = make_float4(a0, a1, a2, a3);
      } else {
        atomicAdd(&d.dq[g].x, a0);
        atomicAdd(&d.dq[g].y, a1);
        atomicAdd(&d.dq[g].z, a2);
        atomicAdd(&d.dq[g].w, a3);
      }
    }
    rec = rec_next;
  }
  if (mark) mark_step_if_last(d);
}

// ------------------------------------------------------------------------------------------------
// Container: coverage of every pixel by the container rings (nonzero rule), once per level.
// Ring vertices are brought into the tile's frame in double and rounded once.
// ------------------------------------------------------------------------------------------------
template <int T, int NT>
__global__ void __launch_bounds__(NT) k_container(Dev d) {
  constexpr int NP = T * T, PPT = NP / NT;
  __shared__ float4 s_seg[kSegCap];
  __shared__ float2 s_seg2[kSegCap];
  const float inv_rho = 1.0f / d.L.rho_px;
  for (int tile = blockIdx.x; tile < d.total_tiles; tile += gridDim.x) {
    const int p = find_prob(d.prob_tile_base, d.n_probs, tile);
    const int lt = tile - d.prob_tile_base[p], ntx = d.prob_ntx[p], res = d.prob_res[p];
    const int tx = lt % ntx, ty = lt / ntx;
    const double ox = (double)(tx * T), oy = (double)(ty * T);
    SegQuery Q[PPT];
    float dx[PPT], dy[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int local = threadIdx.x + k * NT;
      dx[k] = (float)(local % T) + 0.5f;
      dy[k] = (float)(local / T) + 0.5f;
      Q[k].best = FLT_MAX;
      Q[k].idx = 0;
      Q[k].wn = 0;
    }
    const int r0 = d.prob_ring_base[p], r1 = d.prob_ring_base[p + 1];
    for (int r = r0; r < r1; ++r) {
      const int b0 = d.ring_off[r], nv = d.ring_off[r + 1] - b0;
      for (int c0 = 0; c0 < nv; c0 += kSegCap) {
        const int cn = min(kSegCap, nv - c0);
        if (c0 > 0 && threadIdx.x == 0 && d.paths) atomicAdd(&d.paths[3], 1ull);
        __syncthreads();
        for (int j = threadIdx.x; j < cn; j += NT) {
          const int ai = b0 + c0 + j, bi = b0 + (c0 + j + 1) % nv;
          const double ax = d.ring_pts[2 * ai] * res - ox, ay = d.ring_pts[2 * ai + 1] * res - oy;
          const double bx = d.ring_pts[2 * bi] * res - ox, by = d.ring_pts[2 * bi + 1] * res - oy;
          const float fax = (float)ax, fay = (float)ay;
          const float ex = (float)(bx - ax), ey = (float)(by - ay);
          const float ee = ex * ex + ey * ey;
          s_seg[j] = make_float4(fax, fay, ex, ey);
          s_seg2[j] = make_float2((float)by, ee > 0.0f ? 1.0f / ee : 0.0f);
        }
        __syncthreads();
        for (int j = 0; j < cn; ++j) {
          const float4 s = s_seg[j];
          const float2 s2 = s_seg2[j];
#pragma unroll
          for (int k = 0; k < PPT; ++k) seg_update(Q[k], dx[k], dy[k], s, s2, j, true);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int local = threadIdx.x + k * NT;
      const int X = tx * T + local % T, Y = ty * T + local / T;
      if (X >= res || Y >= res) continue;
      const float dist = sqrtf(Q[k].best);
      const float sd = Q[k].wn != 0 ? dist : -dist;
      d.covc[d.prob_pix_base[p] + (long long)Y * res + X] = Sfun(sd * inv_rho);
    }
  }
}

// ------------------------------------------------------------------------------------------------
template <int T>
struct TileCfg;
template <>
struct TileCfg<8> {
  static constexpr int NT = 64;
};
template <>
struct TileCfg<16> {
  static constexpr int NT = 256;
};

template <int T>
static cudaError_t fwd_t(const Dev& d, cudaStream_t s, int pair_grid, int tile_grid, float* bw,
                         float* tau, int part) {
  constexpr int NT = TileCfg<T>::NT;
  cudaError_t e = cudaSuccess;
  if (part & 1) e = klaunch(d.pdl, k_pair_sd<T, NT>, pair_grid, NT, 0, s, d);
  if (e == cudaSuccess && (part & 2))
    e = klaunch(d.pdl, k_composite<T>, tile_grid, kCompWarps * 32, 0, s, d, bw, tau);
  return e;
}

cudaError_t launch_raster_fwd(const Dev& d, cudaStream_t s, int pair_grid, int tile_grid,
                              float* out_bw, float* out_tau, int part) {
  switch (d.tile) {
    case 8: return fwd_t<8>(d, s, pair_grid, tile_grid, out_bw, out_tau, part);
    case 16: return fwd_t<16>(d, s, pair_grid, tile_grid, out_bw, out_tau, part);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_raster_bwd(const Dev& d, cudaStream_t s, int pair_grid, bool mark_step) {
  const int mk = mark_step ? 1 : 0;
  switch (d.tile) {
    case 8:
      return klaunch(d.pdl, d.fit ? k_raster_bwd<8, true> : k_raster_bwd<8, false>, pair_grid,
                     kPairWarps * 32, 0, s, d, mk);
    case 16:
      return klaunch(d.pdl, d.fit ? k_raster_bwd<16, true> : k_raster_bwd<16, false>, pair_grid,
                     kPairWarps * 32, 0, s, d, mk);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_container(const Dev& d, cudaStream_t s) {
  switch (d.tile) {
    case 8: k_container<8, TileCfg<8>::NT><<<d.total_tiles, TileCfg<8>::NT, 0, s>>>(d); break;
    case 16: k_container<16, TileCfg<16>::NT><<<d.total_tiles, TileCfg<16>::NT, 0, s>>>(d); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int T>
static void per_sm_t(RasterOcc* o) {
  constexpr int NT = TileCfg<T>::NT;
  int a = 1, b = 1, c = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pair_sd<T, NT>, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_raster_bwd<T, false>, kPairWarps * 32, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_composite<T>, kCompWarps * 32, 0);
  o->fwd_per_sm = a > 0 ? a : 1;
  o->bwd_per_sm = b > 0 ? b : 1;
  o->tile_per_sm = c > 0 ? c : 1;
  o->bwd_pairs_per_block = kPairWarps;
  o->tiles_per_block = kCompWarps;
}

void raster_occupancy(int tile, RasterOcc* o) {
  if (tile == 16) per_sm_t<16>(o);
  else per_sm_t<8>(o);
}

}  // namespace collage
