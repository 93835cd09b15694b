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
constexpr int kRowCross = 16;   // crossings listed per pixel row of an emission chunk
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

// Winding number of a point (element frame) over every segment of an outline: the crossing test of
// the per-row lists below applied to all segments (for rows that cross the outline too often).
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

// ------------------------------------------------------------------------------------------------
// Emission and signed distances, one (element, chunk) work item per block at a time.  A chunk is a
// square of up to kChunkPx x kChunkPx pixels of the element's tile rectangle (8 x 8 tiles of 8 px,
// 4 x 4 of 16 px); the transform kernel lists every element's chunks.  Per chunk the block
//  1. takes the pair slot of each of its tiles (the element's slots follow its tile rectangle
//     row-major from the base the transform allocated) and records it in the tile's list (a
//     list beyond its capacity latches a status bit: the host grows the lists and runs again);
//  2. passes once over the element's segments, staging them in shared memory by index: a segment
//     whose box meets a tile's pixel-centre box grown by the coverage margin m = rho + pad
//     (+ stroke half-width) (+ 0.06 px of slack) is near that tile (a bit per segment and tile);
//     for every pixel row of the chunk that a segment crosses (half-open in y, on the dy the
//     pixels form) the crossing x is listed for the row, or, when it lies right of every pixel of
//     the chunk, added to the row's backdrop (+1 upward, -1 downward);
//  3. classifies the tiles: a tile that no segment is near has saturated coverage on every pixel
//     (0 or 1, as the winding number of its first pixel says) and needs no per-pixel work;
//  4. its warps take the near tiles one at a time: per pixel, the minimum squared distance over
//     the tile's near segments in index order (the lowest index wins ties, as the oracle's scan
//     does); winding = row backdrop + listed crossings right of the pixel (a row with more than
//     kRowCross crossings tests every segment); sd = +-distance within the margin, else +-1e30
//     (saturated); the (sd, closest segment) record is saved and pairs with a non-saturated pixel
//     are listed for the adjoint.
// Outlines of more than kStageSegs segments are not staged: their tiles test every segment's box
// on the fly, reading the outline from global memory.
// A pixel beyond the margin from every segment near its tile is beyond it from all segments (the
// near test is conservative), so the distance minimum over the near ones is exact wherever it
// matters, and the winding counts every crossing right of the pixel exactly once.
// ------------------------------------------------------------------------------------------------
constexpr int kStageSegs = 512;   // outline segments staged in shared memory
constexpr int kLiveBatch = 32;

// Tiles of the chunk whose grown pixel-centre box a segment's box [x0, x1] x [y0, y1] (absolute
// px) meets: columns [*c0, *c1], rows [*r0, *r1] relative to the chunk origin, clipped to it.
__device__ __forceinline__ void seg_tiles(float x0, float x1, float y0, float y1, float m, int T,
                                          int tx0, int ty0, int ctw, int cth, int* c0, int* c1,
                                          int* r0, int* r1) {
  const float fT = (float)T, iT = 1.0f / fT;  // T is a power of two: x * (1 / T) is x / T exactly
  *c0 = max((int)floorf((x0 - m - (fT - 0.5f)) * iT) + 1 - tx0, 0);
  *c1 = min((int)floorf((x1 + m - 0.5f) * iT) - tx0, ctw - 1);
  *r0 = max((int)floorf((y0 - m - (fT - 0.5f)) * iT) + 1 - ty0, 0);
  *r1 = min((int)floorf((y1 + m - 0.5f) * iT) - ty0, cth - 1);
}

// Squared distance from (dx, dy) to the segment a + u e, u in [0, 1], with f = e / |e|^2 (the
// clamped parameter is then a dot product): the operations of the oracle's closest-point rule.
__device__ __forceinline__ float seg_d2(float dx, float dy, float4 s, float2 f) {
  const float wx = dx - s.x, wy = dy - s.y;
  const float t = __saturatef(fmaf(wy, f.y, wx * f.x));
  const float qx = fmaf(-t, s.z, wx), qy = fmaf(-t, s.w, wy);
  return fmaf(qx, qx, qy * qy);
}

// NT threads per block (128 or 256, the autotuner's choice); registers capped so that 1024
// threads (T = 8) or 512 (T = 16, eight pixels per lane) are resident per SM.
template <int T, int NT>
__global__ void __launch_bounds__(NT, (T == 8 ? 1024 : 512) / NT) k_raster_chunks(Dev d) {
  pdl_enter();
  constexpr int CW = kChunkPx / T, NCT = CW * CW, NP = T * T, PPL = NP / 32;
  constexpr int ROWS = kChunkPx, MW = kStageSegs / 32;
  __shared__ float4 s_seg[kStageSegs];  // start (px, relative to the translation), direction
  __shared__ float2 s_f[kStageSegs];    // direction / |direction|^2
  __shared__ unsigned s_mask[NCT][MW];  // bit j of tile k: segment j is near tile k
  __shared__ int s_slot[NCT];           // pair slot of each tile (-1: void)
  __shared__ unsigned char s_tn[NCT];   // some segment is near the tile
  __shared__ int2 s_ntile[NCT];         // the near tiles: (pair slot, tile | column << 8 | row << 16)
  __shared__ int2 s_row[ROWS];          // per pixel row: (crossings right of every pixel, listed)
  __shared__ float2 s_rx[ROWS][kRowCross];  // listed crossings: (x, +1 upward / -1 downward)
  __shared__ int s_nt, s_take;
  __shared__ int s_next[2];
  __shared__ int4 s_live[kLiveBatch];
  __shared__ int s_nlive;
  const float inv_rho = 1.0f / d.L.rho_px, pad = d.L.pad_px;
  const int tid = threadIdx.x, lane = tid & 31;
  const int n_heavy = d.chunk_count[0], n_chunks = n_heavy + d.chunk_count[1];
  if (blockIdx.x == 0 && tid == 0) {
    // the transform has completed: its slot count becomes the iteration's pair count, its
    // pending-step flag is spent, and the composite's fullest-tile maximum starts over
    *d.total_pairs = *d.pair_need;
    *d.pair_need = 0;
    *d.tile_max = 0;
    *d.pending = 0;
  }
  // the slots are void when the pairs exceed the capacity (the transform latched it)
  for (int i = (*d.status & kStatusOverflow) ? n_chunks : blockIdx.x, it = 0; i < n_chunks; ++it) {
    if (tid == 0) {
      // chunks beyond the grid are taken by an atomic count (none when the grid covers them all)
      s_next[it & 1] = n_chunks > (int)gridDim.x ? (int)gridDim.x + atomicAdd(&d.work[0], 1) : n_chunks;
      s_nlive = 0;
      s_take = 0;
    }
    const int li = i < n_heavy ? i : d.list_cap - 1 - (i - n_heavy);
    if (!in_bounds(d, li >= 0 && li < d.list_cap)) break;
    const int4 rec = d.near_list[li];
    const int g = rec.x, tx0 = rec.y & 0xffff, ty0 = rec.y >> 16, p = rec.z;
    if (!in_bounds(d, g >= 0 && g < d.n_elems && p >= 0 && p < d.n_probs)) break;
    const int4 r = d.rect[g];
    const int cs = min(d.chunk_tiles, CW);
    const int ctw = min(cs, r.z - tx0 + 1), cth = min(cs, r.w - ty0 + 1), nct = ctw * cth;
    const int res = d.prob_res[p], ntx = d.prob_ntx[p], tb = d.prob_tile_base[p];
    const int v0 = d.elem_voff[g], nv = d.elem_voff[g + 1] - v0;
    const bool closed = d.elem_closed[g] != 0;
    const int ns = closed ? nv : nv - 1;
    const bool staged = ns <= kStageSegs;
    const int mw = staged ? (ns + 31) >> 5 : 0;
    // 1. pair slots; cleared marks and row lists
    if (tid < NCT) {
      int slot = -1;
      const int t = tb + (ty0 + tid / ctw) * ntx + tx0 + tid % ctw;
      if (tid < nct && in_bounds(d, t >= tb && t < d.prob_tile_base[p + 1])) {
        const int u = d.elem_pbase[g] + (ty0 + tid / ctw - r.y) * (r.z - r.x + 1) + tx0 + tid % ctw - r.x;
        if (in_bounds(d, u >= 0 && u < d.cap)) {
          slot = u;
          d.pair_elem[slot] = g;
          const int k = atomicAdd(&d.tile_n[t], 1);
          if (k < d.tile_cap) d.tile_list[(size_t)t * d.tile_cap + k] = slot;
          else atomicOr(d.status, kStatusTileCap);
        }
      }
      s_slot[tid] = slot;
      s_tn[tid] = 0;
    }
    for (int q = tid; q < nct * mw; q += NT) s_mask[q / mw][q % mw] = 0u;
    for (int q = tid; q < ROWS; q += NT) s_row[q] = make_int2(0, 0);
    const float4 tp = d.tpx[g], bb = d.bbox[g];
    const float hwpx = closed ? 0.0f : d.elem_hw[g] * (float)res;
    const float mrg = d.L.rho_px + pad + hwpx, mrg2 = mrg * mrg;
    const float tpx = tp.x + tp.z, tpy = tp.y + tp.w;
    const int X0 = tx0 * T, Y0 = ty0 * T, ncol = ctw * T, nrow = cth * T;
    // the chunk's pixel-centre box in the element frame, as the pixels form dx and dy
    const float min_dx = ((float)X0 + 0.5f - tp.x) - tp.z;
    const float max_dx = ((float)(X0 + ncol - 1) + 0.5f - tp.x) - tp.z;
    const float sl = mrg + 0.06f;  // near test margin with slack
    __syncthreads();
    // 2. one pass over the segments: staging, the tiles they are near, row crossings
    if (ns > kStageSegs && tid == 0 && d.paths) atomicAdd(&d.paths[1], 1ull);
    for (int j = tid; j < ns; j += NT) {
      const float4 sa = d.segA[v0 + j];
      const float2 sb = d.segB[v0 + j];
      if (staged) {
        s_seg[j] = sa;
        s_f[j] = make_float2(sa.z * sb.y, sa.w * sb.y);
      }
      const float bx = sa.x + sa.z, by = sb.x;
      const float x0 = fminf(sa.x, bx), x1 = fmaxf(sa.x, bx), y0 = fminf(sa.y, by), y1 = fmaxf(sa.y, by);
      int c0, c1, r0, r1;
      seg_tiles(x0 + tpx, x1 + tpx, y0 + tpy, y1 + tpy, sl, T, tx0, ty0, ctw, cth, &c0, &c1, &r0, &r1);
      for (int rr = r0; rr <= r1; ++rr)
        for (int cc = c0; cc <= c1; ++cc) {
          if (!in_bounds(d, rr * ctw + cc < NCT)) continue;
          s_tn[rr * ctw + cc] = 1;
          if (staged) atomicOr(&s_mask[rr * ctw + cc][j >> 5], 1u << (j & 31));
        }
      if (closed && y1 > y0 && x1 > min_dx) {  // crosses some row right of the first pixel column
        // candidate rows (one row of slack each side), then the exact half-open test
        const int q0 = max((int)floorf(y0 + tpy - 0.5f) - Y0 - 1, 0);
        const int q1 = min((int)ceilf(y1 + tpy - 0.5f) - Y0 + 1, nrow - 1);
        const float slope = d.segS[v0 + j];
        for (int q = q0; q <= q1; ++q) {
          if (!in_bounds(d, q < ROWS)) break;
          const float yr = ((float)(Y0 + q) + 0.5f - tp.y) - tp.w;
          const bool a_le = yr - sa.y >= 0.0f, b_le = yr - by >= 0.0f;
          if (a_le == b_le) continue;
          const float xc = fmaf(yr - sa.y, slope, sa.x);
          const int dir = a_le ? 1 : -1;
          if (xc > max_dx) {
            atomicAdd(&s_row[q].x, dir);  // right of every pixel of the row
          } else if (xc > min_dx) {
            const int k = atomicAdd(&s_row[q].y, 1);
            if (k < kRowCross) s_rx[q][k] = make_float2(xc, (float)dir);
          }
        }
      }
    }
    __syncthreads();
    // 3. classification; the near tiles in tile order
    if (tid < nct && s_slot[tid] >= 0) {
      const int slot = s_slot[tid];
      uint8_t cls = kPairNear;
      if (!s_tn[tid]) {
        int w = 0;
        if (closed) {
          const int q = (tid / ctw) * T;
          const float dx0 = ((float)(X0 + (tid % ctw) * T) + 0.5f - tp.x) - tp.z;
          const int2 row = s_row[q];
          if (row.y <= kRowCross) {
            float wf = (float)row.x;
            for (int k = 0; k < row.y; ++k) {
              const float2 c = s_rx[q][k];
              if (dx0 < c.x) wf += c.y;
            }
            w = (int)wf;
          } else {
            w = winding_all(d, v0, ns, dx0, ((float)(Y0 + q) + 0.5f - tp.y) - tp.w);
          }
        }
        cls = w != 0 ? kPairIn : kPairOut;
        if (d.deterministic) d.partial[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      d.pair_cls[slot] = cls;
    }
    if (tid < 32) {  // warp 0: the near tiles, in tile order
      int n = 0;
      for (int k0 = 0; k0 < nct; k0 += 32) {
        const int k = k0 + lane;
        const bool nr = k < nct && s_slot[k] >= 0 && s_tn[k];
        const unsigned bal = __ballot_sync(0xffffffffu, nr);
        if (nr) s_ntile[n + __popc(bal & ((1u << lane) - 1u))] = make_int2(s_slot[k], k | (k % ctw) << 8 | (k / ctw) << 16);
        n += __popc(bal);
      }
      if (lane == 0) s_nt = n;
    }
    __syncthreads();
    const int nt = s_nt;
    // 4. the near tiles, one per warp at a time (the next one taken while this one is worked on)
    int ni = 0;
    if (lane == 0) ni = atomicAdd(&s_take, 1);
    ni = __shfl_sync(0xffffffffu, ni, 0);
    while (ni < nt) {
      int nn = 0;
      if (lane == 0) nn = atomicAdd(&s_take, 1);
      const int2 nti = s_ntile[ni];
      const int slot = nti.x, k = nti.y & 0xff, kr = nti.y >> 16;
      const int tcx = tx0 + ((nti.y >> 8) & 0xff), tcy = ty0 + kr;
      float dx[PPL], dy[PPL], best[PPL];
      int bidx[PPL];
#pragma unroll
      for (int e = 0; e < PPL; ++e) {
        const int local = lane + 32 * e;
        dx[e] = ((float)(tcx * T + local % T) + 0.5f - tp.x) - tp.z;
        dy[e] = ((float)(tcy * T + local / T) + 0.5f - tp.y) - tp.w;
        best[e] = FLT_MAX;
        bidx[e] = 0;
      }
      if (staged) {
        for (int w = 0; w < mw; ++w) {
          unsigned bits = s_mask[k][w];
          while (bits) {
            const int j = w * 32 + __ffs(bits) - 1;  // in index order
            bits &= bits - 1u;
            const float4 sg = s_seg[j];
            const float2 f = s_f[j];
#pragma unroll
            for (int e = 0; e < PPL; ++e) {
              const float d2 = seg_d2(dx[e], dy[e], sg, f);
              if (d2 < best[e]) {
                best[e] = d2;
                bidx[e] = j;
              }
            }
          }
        }
      } else {
        // the tile's near segments by the same box test as the marks, from global memory
        const int kc = k % ctw, kr = k / ctw;
        for (int j = 0; j < ns; ++j) {
          const float4 s = d.segA[v0 + j];
          const float2 sb = d.segB[v0 + j];
          const float bx = s.x + s.z;
          int c0, c1, r0, r1;
          seg_tiles(fminf(s.x, bx) + tpx, fmaxf(s.x, bx) + tpx, fminf(s.y, sb.x) + tpy,
                    fmaxf(s.y, sb.x) + tpy, sl, T, tx0, ty0, ctw, cth, &c0, &c1, &r0, &r1);
          if (kc < c0 || kc > c1 || kr < r0 || kr > r1) continue;
          const float2 f = make_float2(s.z * sb.y, s.w * sb.y);
#pragma unroll
          for (int e = 0; e < PPL; ++e) {
            const float d2 = seg_d2(dx[e], dy[e], s, f);
            if (d2 < best[e]) {
              best[e] = d2;
              bidx[e] = j;
            }
          }
        }
      }
      float2* sv = d.saved + (size_t)slot * NP;
      bool live = false;
#pragma unroll
      for (int e = 0; e < PPL; ++e) {
        const int local = lane + 32 * e;
        const int X = tcx * T + local % T, Y = tcy * T + local / T;
        const bool act = X < res && Y < res && dx[e] >= bb.x && dx[e] <= bb.z && dy[e] >= bb.y &&
                         dy[e] <= bb.w;
        float sd = -kFar;
        if (act) {
          int w = 0;
          if (closed) {
            const int q = Y - Y0;
            const int2 row = s_row[q];
            if (row.y <= kRowCross) {
              float wf = (float)row.x;
              for (int c = 0; c < row.y; ++c) {
                const float2 cr = s_rx[q][c];
                if (dx[e] < cr.x) wf += cr.y;
              }
              w = (int)wf;
            } else {
              w = winding_all(d, v0, ns, dx[e], dy[e]);
            }
          }
          if (best[e] < mrg2) {
            const float dist = sqrtf(best[e]);
            sd = closed ? (w != 0 ? dist : -dist) : hwpx - dist;
          } else {
            sd = (closed && w != 0) ? kFar : -kFar;
          }
          live |= fabsf(sd * inv_rho) < 1.0f || fabsf((sd + pad) * inv_rho) < 1.0f;
        }
        sv[local] = make_float2(sd, __int_as_float(bidx[e]));
      }
      if (d.paths && closed && lane < T && s_row[kr * T + lane].y > kRowCross)
        atomicAdd(&d.paths[0], 1ull);
      if (__any_sync(0xffffffffu, live)) {
        if (lane == 0) {
          const int4 lr = make_int4(slot, g, tcx | (tcy << 16), p);
          const int q = atomicAdd(&s_nlive, 1);
          if (q < kLiveBatch) {
            s_live[q] = lr;
          } else {
            const int at = atomicAdd(&d.work[1], 1);
            if (in_bounds(d, at < d.cap)) d.live_list[at] = lr;
          }
        }
      } else if (lane == 0 && d.deterministic) {
        d.partial[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      ni = __shfl_sync(0xffffffffu, nn, 0);
    }
    __syncthreads();
    // the chunk's live pairs go out with one atomic
    if (tid < 32) {
      const int n = min(s_nlive, kLiveBatch);
      int at = 0;
      if (lane == 0 && n > 0) at = atomicAdd(&d.work[1], n);
      at = __shfl_sync(0xffffffffu, at, 0);
      if (lane < n && in_bounds(d, at + lane < d.cap)) d.live_list[at + lane] = s_live[lane];
    }
    __syncthreads();  // s_live, s_nlive and the shared lists are reused by the next chunk
    i = s_next[it & 1];
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
constexpr int kCompGroup = 4;   // pairs whose records are read together
constexpr int kCompWide = 256;  // lists up to this long are ranked from shared memory
template <int T>
__global__ void __launch_bounds__(kCompWarps * 32) k_composite(Dev d, float* out_bw, float* out_tau) {
  pdl_enter();
  constexpr int NP = T * T, PPL = NP / 32;
  __shared__ int s_slot[kCompWarps][32];
  __shared__ uint8_t s_cls[kCompWarps][32];
  __shared__ int s_wide[kCompWarps][kCompWide];  // a long list's element ids, in list order
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // the emission has completed: its work list is spent
    d.chunk_count[0] = d.chunk_count[1] = 0;
    d.work[0] = 0;
  }
  if (*d.status & kStatusNoBins) return;
  const float inv_rho = 1.0f / d.L.rho_px, pad = d.L.pad_px, tau = d.L.tau;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int* w_slot = s_slot[wid];
  uint8_t* w_cls = s_cls[wid];
  __shared__ int s_mmax;
  if (threadIdx.x == 0) s_mmax = 0;
  __syncthreads();
  int m_max = 0;  // the fullest list this warp saw (the host keeps the lists' capacity ahead of it)
  for (int tile = blockIdx.x * kCompWarps + wid; tile < d.total_tiles; tile += gridDim.x * kCompWarps) {
    int p, tx, ty, res;
    tile_coords(d, tile, T, p, tx, ty, res);
    const long long pixbase = d.prob_pix_base[p];
    // the tile's pairs (emission order) and, for the next iteration, an empty list; the count and
    // the first list entries are read together (an entry is used only below the count, and the
    // slot it names is clamped into the buffer before its element and class are read)
    const size_t lb = (size_t)tile * d.tile_cap;
    int m = d.tile_n[tile];
    const int sl0 = lane < d.tile_cap ? d.tile_list[lb + lane] : 0;
    // the container coverage of the lane's pixels (independent of the pairs)
    float cov[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int local = lane + 32 * k;
      const int X = min(tx * T + local % T, res - 1), Y = min(ty * T + local / T, res - 1);
      cov[k] = d.covc[pixbase + (long long)Y * res + X];
    }
    if (!in_bounds(d, m >= 0 && m <= d.tile_cap)) m = 0;
    m_max = max(m_max, m);
    __syncwarp();  // the previous tile's readers of this warp's lists and of tile_n are done
    if (lane == 0) {
      d.tile_n[tile] = 0;
      d.tile_m[tile] = m;
    }
    const bool small = m <= 32;
    int* sorted = d.tile_sorted + lb;
    int* sorted_slot = d.tile_sorted_slot + lb;
    if (small) {
      const int sl = (unsigned)sl0 < (unsigned)d.cap ? sl0 : 0;
      const int v0 = d.pair_elem[sl];
      const uint8_t c0 = d.pair_cls[sl];
      const int v = lane < m ? v0 : 0;
      int r = 0;
      for (int j = 0; j < m; ++j) r += __shfl_sync(0xffffffffu, v, j) < v ? 1 : 0;
      if (lane < m) {
        w_slot[r] = sl;
        w_cls[r] = c0;
        sorted[r] = v;
        sorted_slot[r] = sl;
      }
    } else if (m <= kCompWide) {
      // the element ids read once (independent loads), then each entry ranked against them all
      if (lane == 0 && d.paths) atomicAdd(&d.paths[2], 1ull);
      int* wv = s_wide[wid];
      for (int i = lane; i < m; i += 32) wv[i] = d.pair_elem[d.tile_list[lb + i]];
      __syncwarp();
      for (int i = lane; i < m; i += 32) {
        const int vi = wv[i];
        int r = 0;
        for (int j = 0; j < m; ++j) r += wv[j] < vi ? 1 : 0;  // one address for every lane
        sorted[r] = vi;
        sorted_slot[r] = d.tile_list[lb + i];
      }
    } else {
      if (lane == 0 && d.paths) atomicAdd(&d.paths[2], 1ull);
      for (int i = lane; i < m; i += 32) {
        const int si = d.tile_list[lb + i], vi = d.pair_elem[si];
        int r = 0;
        for (int j = 0; j < m; ++j) r += d.pair_elem[d.tile_list[lb + j]] < vi ? 1 : 0;
        sorted[r] = vi;
        sorted_slot[r] = si;
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
    // in groups of kCompGroup pairs whose signed distances are read before any is used
    for (int i0 = 0; i0 < m; i0 += kCompGroup) {
      float sd[kCompGroup][PPL];
      uint8_t cls[kCompGroup];
#pragma unroll
      for (int u = 0; u < kCompGroup; ++u) {
        const int i = i0 + u;
        cls[u] = kPairOut;
        if (i < m) {
          const int slot = small ? w_slot[i] : sorted_slot[i];
          cls[u] = small ? w_cls[i] : d.pair_cls[slot];
#pragma unroll
          for (int k = 0; k < PPL; ++k)  // an inside pair has c = c^pad = 1: sd = +1e30 gives that
            sd[u][k] = cls[u] == kPairNear ? d.saved[(size_t)slot * NP + lane + 32 * k].x : kFar;
        }
      }
#pragma unroll
      for (int u = 0; u < kCompGroup; ++u) {
        if (cls[u] == kPairOut) continue;  // c = c^pad = 0: factors of 1
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
          const float x = sd[u][k] * inv_rho;
          const float omc = Sfun(-x), cp = Sfun((sd[u][k] + pad) * inv_rho);
          if (omc == 0.0f) zc[k] += 1;
          else keep[k] *= omc;
          keept[k] *= 1.0f - tau * cp;
          nfull[k] += cp == 1.0f;
          partial[k] |= cp > 0.0f && cp < 1.0f;
        }
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
      const float W = cov[k] >= 0.5f ? d.L.w_in : d.L.w_out;
      const float df = ihat - (1.0f - cov[k]);
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
  if (lane == 0) atomicMax(&s_mmax, m_max);
  __syncthreads();
  if (threadIdx.x == 0 && s_mmax > 0) atomicMax(d.tile_max, s_mmax);
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
  if (*d.status & kStatusNoBins) return;
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
    if (!in_bounds(d, slot >= 0 && slot < d.cap && g >= 0 && g < d.n_elems && p >= 0 && p < d.n_probs)) {
      rec = rec_next;
      continue;
    }
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
      if (gsd[k] != 0.0f && !in_bounds(d, (unsigned)__float_as_int(srec[k].y) <
                                               (unsigned)(d.elem_voff[g + 1] - v0)))
        gsd[k] = 0.0f;
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
  cudaError_t e = cudaSuccess;
  if (part & 1)
    e = d.emit_threads == 256 ? klaunch(d.pdl, k_raster_chunks<T, 256>, pair_grid, 256, 0, s, d)
                              : klaunch(d.pdl, k_raster_chunks<T, 128>, pair_grid, 128, 0, s, d);
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
static void per_sm_t(int emit_threads, RasterOcc* o) {
  int a = 1, b = 1, c = 1;
  if (emit_threads == 256) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_raster_chunks<T, 256>, 256, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_raster_chunks<T, 128>, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_raster_bwd<T, false>, kPairWarps * 32, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_composite<T>, kCompWarps * 32, 0);
  o->fwd_per_sm = a > 0 ? a : 1;
  o->bwd_per_sm = b > 0 ? b : 1;
  o->tile_per_sm = c > 0 ? c : 1;
  o->bwd_pairs_per_block = kPairWarps;
  o->tiles_per_block = kCompWarps;
}

void raster_occupancy(int tile, int emit_threads, RasterOcc* o) {
  if (tile == 16) per_sm_t<16>(emit_threads, o);
  else per_sm_t<8>(emit_threads, o);
}

}  // namespace collage
