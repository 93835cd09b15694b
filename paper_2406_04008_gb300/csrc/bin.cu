// Transform (Eq. 2) and tile binning.
//
// Binning: the transform kernel gives every element a block of consecutive pair slots, one per tile
// of its tile rectangle (one atomic per element; a total beyond the capacity latches the overflow
// bit before any pair is written), and lists every element's kChunkPx-square chunks of its
// rectangle; the emission (csrc/raster.cu, per chunk) records each (tile, element) pair's slot in
// its tile's list; the composite then orders each tile's short list by element id before using it,
// so every tile lists its elements in increasing order whatever the order of the atomics.  The tile rectangle follows a fixed float formula
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

// Vertex of an element relative to its translation, in pixels: (s res R(theta)) v.  The matrix is
// formed in double once per element and split into float hi + lo parts; the per-vertex product uses
// error-free transformations in float (FMA two-product and Knuth's two-sum, as in Ogita, Rump &
// Oishi 2005), so the result is within about one float ulp of the exact value without FP64 work
// per vertex (FP64 throughput is low on this part).  Explicit round-to-nearest intrinsics keep the
// compiler from contracting the error terms away.  A segment's end point and the next segment's
// start point come from the same call, so they are bitwise equal (the winding test relies on it).
struct RotFF {
  float m[4][2];  // row-major 2x2, (hi, lo)
};

__device__ __forceinline__ float dot2_ff(const float (&a)[2], const float (&b)[2], float vx, float vy) {
  const float p1 = __fmul_rn(a[0], vx), e1 = __fmaf_rn(a[0], vx, -p1);
  const float p2 = __fmul_rn(b[0], vy), e2 = __fmaf_rn(b[0], vy, -p2);
  const float sum = __fadd_rn(p1, p2);
  const float bb = __fsub_rn(sum, p1);
  const float es = __fadd_rn(__fsub_rn(p1, __fsub_rn(sum, bb)), __fsub_rn(p2, bb));
  const float tail = __fmaf_rn(a[1], vx, __fmaf_rn(b[1], vy, __fadd_rn(__fadd_rn(e1, e2), es)));
  return __fadd_rn(sum, tail);
}

__device__ __forceinline__ float2 vertex_px(const float2 v, const RotFF& M) {
  return make_float2(dot2_ff(M.m[0], M.m[1], v.x, v.y), dot2_ff(M.m[2], M.m[3], v.x, v.y));
}

// One block per element: the pending Adam step of the previous iteration, then segment records
// (start, direction, end y, 1/|e|^2) of the vertices relative to the translation, translation in
// pixels as a float hi/lo pair, outline box grown by the coverage margin, tile rectangle, the
// element's pair slots and its emission chunks.
// Threads 0..3 each take the step in registers (the same arithmetic), write back one parameter and
// form one entry of the rotation-scale matrix, so one barrier separates the step from the vertices.
// Warps 0..2 then transform the vertices (lanes own consecutive vertices; a segment's end point is
// the next lane's start point, shuffled, so each vertex is transformed once) while warp 3 files the
// tile rectangle, the pair slots and the chunk list, which do not depend on the vertices.
constexpr int kTfThreads = 128;
constexpr int kTfVertexWarps = 3;
__global__ void __launch_bounds__(kTfThreads) k_transform(Dev d, int zero_grad) {
  pdl_enter();
  __shared__ RotFF s_rot;
  __shared__ float4 s_q;
  __shared__ float s_box[4][kTfVertexWarps];
  const int g = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // (a single problem's resolution is read without waiting for the element's problem index)
  const int p = d.n_probs == 1 ? 0 : d.elem_prob[g];
  const int res = d.prob_res[p];
  if (g == 0 && threadIdx.x == 0) {  // this iteration's live pairs and finished gradient blocks
    d.work[1] = 0;
    d.work[3] = 0;
  }
  // the outline and its first vertices do not depend on the step: read before the barrier
  const int v0 = d.elem_voff[g], nv = d.elem_voff[g + 1] - v0;
  const bool closed = d.elem_closed[g] != 0;
  const float hw = closed ? 0.0f : d.elem_hw[g];
  const float rbin = wid == kTfVertexWarps ? d.elem_rbin[g] : 0.0f;
  const int k_first = wid * 32 + lane;
  float2 va0 = make_float2(0.f, 0.f), vb0 = make_float2(0.f, 0.f);
  if (wid < kTfVertexWarps && k_first < nv) {
    va0 = d.vloc[v0 + k_first];
    if (lane == 31 || k_first + 1 == nv) vb0 = d.vloc[v0 + (k_first + 1 == nv ? 0 : k_first + 1)];
  }
  if (threadIdx.x < 4) {
    const int k = threadIdx.x;
    float4 q = d.q[g], m, v;
    // the previous iteration's step (when the outlines are fitted the transforms stay fixed)
    const bool step = *d.pending && !d.fit;
    if (step) {
      m = d.m[g];
      v = d.v[g];
      const uchar4 tr = d.trainable ? d.trainable[g] : make_uchar4(1, 1, 1, 1);
      adam_apply(d, *d.step, d.dq[g], tr, q, m, v);
    }
    // the host-buffer step: the caller's params replace the stepped ones (the moments keep the step)
    if (d.q_in) q = d.q_in[g];
    __syncwarp(0xfu);  // every reader of the old params is done
    auto pick = [k](float4 x) { return k == 0 ? x.x : k == 1 ? x.y : k == 2 ? x.z : x.w; };
    if (step) {
      reinterpret_cast<float*>(d.m + g)[k] = pick(m);
      reinterpret_cast<float*>(d.v + g)[k] = pick(v);
    }
    if (step || d.q_in) reinterpret_cast<float*>(d.q + g)[k] = pick(q);
    if (k == 0) s_q = q;
    double sn, c;
    sincos((double)q.z, &sn, &c);
    const double sc = (double)q.w * (double)res;
    const double mk = k == 0 ? sc * c : k == 1 ? -sc * sn : k == 2 ? sc * sn : sc * c;
    const float hi = (float)mk;
    s_rot.m[k][0] = hi;
    s_rot.m[k][1] = (float)(mk - (double)hi);
  }
  __syncthreads();
  const float4 q = s_q;
  if (wid == kTfVertexWarps) {
    // the tile rectangle, the pair slots and the emission's chunks (lane 0 takes the counts)
    const bool finite = isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w) && q.w > 0.0f;
    int4 r = make_int4(0, 0, -1, -1);
    if (finite) r = bin_rect(q, rbin, hw, res, d.tile, d.L.rho_px, d.L.pad_px);
    else if (lane == 0) atomicOr(d.status, kStatusBadParam);
    if (lane == 0) {
      d.rect[g] = r;
      if (zero_grad) d.dq[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (r.z >= r.x && r.w >= r.y) {
      // the pair slots of the rectangle; beyond the capacity the bins of the iteration are void
      const int n = (r.z - r.x + 1) * (r.w - r.y + 1);
      // the emission's work: the rectangle in chunks of kChunkPx / T tiles a side; chunks whose
      // segments x tiles exceed kHeavyChunk are listed from the front, the others from the back,
      // so that the emission takes the costliest first and none trails at the end
      const int cw = d.chunk_tiles, nx = (r.z - r.x) / cw + 1, ny = (r.w - r.y) / cw + 1;
      const int tiles = min(r.z - r.x + 1, cw) * min(r.w - r.y + 1, cw);
      const bool heavy = nv * tiles > kHeavyChunk;
      int pbase = 0, cbase = 0;
      if (lane == 0) {  // both counts taken at once (neither waits for the other's result)
        pbase = atomicAdd(d.pair_need, n);
        cbase = atomicAdd(d.chunk_count + (heavy ? 0 : 1), nx * ny);
        if (pbase > d.cap - n) atomicOr(d.status, kStatusOverflow);
        d.elem_pbase[g] = pbase;
      }
      cbase = __shfl_sync(0xffffffffu, cbase, 0);
      // (heavy + light chunks beyond the list mean more pairs than the capacity too: the iteration
      // overflows and the emission does not read the list; every write stays inside it)
      if (cbase + nx * ny <= d.list_cap)
        for (int c = lane; c < nx * ny; c += 32) {
          const int at = heavy ? cbase + c : d.list_cap - 1 - (cbase + c);
          d.near_list[at] = make_int4(g, (r.x + (c % nx) * cw) | ((r.y + (c / nx) * cw) << 16), p, 0);
        }
    }
    return;  // no barrier follows for this warp
  }
  const RotFF rot = s_rot;
  float xmin = FLT_MAX, ymin = FLT_MAX, xmax = -FLT_MAX, ymax = -FLT_MAX;
  for (int k0 = wid * 32; k0 < nv; k0 += kTfVertexWarps * 32) {  // warp-uniform trip count
    const int k = k0 + lane;
    const bool first = k0 == wid * 32;
    float2 a = make_float2(0.f, 0.f);
    if (k < nv) {
      a = vertex_px(first ? va0 : d.vloc[v0 + k], rot);
      xmin = fminf(xmin, a.x);
      xmax = fmaxf(xmax, a.x);
      ymin = fminf(ymin, a.y);
      ymax = fmaxf(ymax, a.y);
    }
    float2 b;
    b.x = __shfl_down_sync(0xffffffffu, a.x, 1);
    b.y = __shfl_down_sync(0xffffffffu, a.y, 1);
    const int kb = k + 1 == nv ? 0 : k + 1;
    if (k < nv && (lane == 31 || k + 1 == nv)) b = vertex_px(first ? vb0 : d.vloc[v0 + kb], rot);
    if (k < nv) {
      float4 sa = make_float4(a.x, a.y, 0.f, 0.f);
      float2 sb = make_float2(a.y, 0.f);
      float slope = 0.0f;
      if (closed || k + 1 < nv) {
        const float ex = b.x - a.x, ey = b.y - a.y, ee = ex * ex + ey * ey;
        sa.z = ex;
        sa.w = ey;
        sb = make_float2(b.y, ee > 0.0f ? 1.0f / ee : 0.0f);
        slope = ey != 0.0f ? ex / ey : 0.0f;
      }
      d.segA[v0 + k] = sa;
      d.segB[v0 + k] = sb;
      d.segS[v0 + k] = slope;
    }
  }
  xmin = warp_min(xmin);
  ymin = warp_min(ymin);
  xmax = warp_max(xmax);
  ymax = warp_max(ymax);
  if (lane == 0) {
    s_box[0][wid] = xmin;
    s_box[1][wid] = ymin;
    s_box[2][wid] = xmax;
    s_box[3][wid] = ymax;
  }
  // the vertex warps only (warp 3 has left): named barrier 1 over their threads
  asm volatile("bar.sync 1, %0;" ::"n"(kTfVertexWarps * 32) : "memory");
  if (threadIdx.x == 0) {
    for (int w = 1; w < kTfVertexWarps; ++w) {
      xmin = fminf(xmin, s_box[0][w]);
      ymin = fminf(ymin, s_box[1][w]);
      xmax = fmaxf(xmax, s_box[2][w]);
      ymax = fmaxf(ymax, s_box[3][w]);
    }
    const double tx = (double)q.x * res, ty = (double)q.y * res;
    const float hx = (float)tx, hy = (float)ty;
    d.tpx[g] = make_float4(hx, hy, (float)(tx - (double)hx), (float)(ty - (double)hy));
    // outline box relative to the translation, grown by the coverage margin (+ rounding slack)
    const float m = d.L.rho_px + d.L.pad_px + hw * (float)res + 0.01f;
    d.bbox[g] = make_float4(xmin - m, ymin - m, xmax + m, ymax + m);
  }
}

cudaError_t launch_transform(const Dev& d, cudaStream_t s, bool zero_grad) {
  return klaunch(d.pdl, k_transform, d.n_elems, kTfThreads, 0, s, d, zero_grad ? 1 : 0);
}



}  // namespace collage
