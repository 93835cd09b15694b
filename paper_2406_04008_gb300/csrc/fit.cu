// Outline fitting (Sec. 3, Vector Representation): an item is a closed path of cubic Bezier curves
// whose control points are fitted to the item's silhouette by differentiable rendering.  Here the
// points of every element are the parameters: the adjoint leaves dL/d(flattened vertex) in dv
// (element-local unit coordinates), and one block per element maps it to the points through the
// flattening (Bernstein weights of each sample for a cubic path, the identity for polygons and
// polylines), takes an Adam step on the points and flattens the outline again.
#include <cfloat>

#include "internal.h"

namespace collage {

constexpr int kCtrlThreads = 128;

// Bernstein weights of sample j of a curve sampled spc times (t = j / spc, u = 1 - t; u^3, 3u^2 t,
// 3u t^2, t^3), in float: FP64 instructions are slow and long-latency on this part, and the
// vertices are float either way (within an ulp or two of the host's double flattening).
__device__ __forceinline__ void bernstein(int j, int spc, float (&b)[4]) {
  const float t = (float)j / (float)spc, u = 1.0f - t;
  b[0] = u * u * u;
  b[1] = 3.0f * u * u * t;
  b[2] = 3.0f * u * t * t;
  b[3] = t * t * t;
}

constexpr int kBernMax = 256;   // samples per curve whose weights are tabled in shared memory
constexpr int kStageDv = 2048;  // vertex gradients of an element staged in shared memory

// mode 0: dv -> dctrl, dv cleared; 1: the same, then an Adam step on the points (step *d.step,
// the update adam_update makes, without a clamp) and the flattening; 2: the flattening only.
__global__ void __launch_bounds__(kCtrlThreads) k_ctrl_step(Dev d, int mode) {
  pdl_enter();
  __shared__ float s_r[kCtrlThreads / 32];
  __shared__ float s_w[kBernMax][4];  // the Bernstein weights of the samples, formed once
  __shared__ float2 s_dv[kStageDv];    // the element's vertex gradients, read once
  if (mode != 2 && (*d.status & kStatusVoid)) return;  // a void iteration
  const int g = blockIdx.x;
  const int c0 = d.elem_coff[g], np = d.elem_coff[g + 1] - c0;
  const int v0 = d.elem_voff[g], nv = d.elem_voff[g + 1] - v0;
  const bool cubic = d.elem_cubic[g] != 0;
  const int spc = d.spc, ncurve = np / 3;
  const bool table = cubic && spc <= kBernMax;
  if (table) {
    for (int j = threadIdx.x; j < spc; j += kCtrlThreads) {
      float b[4];
      bernstein(j, spc, b);
      for (int r = 0; r < 4; ++r) s_w[j][r] = b[r];
    }
    __syncthreads();
  }
  // weight r of sample j (from the table when there is one)
  auto weight = [&](int j, int r) -> float {
    if (table) return s_w[j][r];
    float b[4];
    bernstein(j, spc, b);
    return b[r];
  };
  if (mode != 2) {
    // the vertex gradients are read (and cleared for the next pass) once, coalesced
    const bool staged = nv <= kStageDv;
    if (staged) {
      for (int i = threadIdx.x; i < nv; i += kCtrlThreads) {
        s_dv[i] = d.dv[v0 + i];
        d.dv[v0 + i] = make_float2(0.0f, 0.0f);
      }
      __syncthreads();
    }
    const float2* dv = staged ? s_dv : d.dv + v0;
    // point k of a cubic path is entry k % 3 of curve k / 3; an anchor (k % 3 = 0) is also entry 3
    // of the previous curve.  A fixed order over the samples: the sums are reproducible given dv.
    const int t = *d.step;
    const float bc1 = 1.0f - powf(d.b1, (float)t), bc2 = 1.0f - powf(d.b2, (float)t);
    const float step_size = d.lr / bc1, bc2s = sqrtf(bc2);
    for (int k = threadIdx.x; k < np; k += kCtrlThreads) {
      float2 gk = make_float2(0.0f, 0.0f);
      if (!cubic) {
        gk = dv[k];
      } else {
        const int c = k / 3, r = k % 3;
        for (int j = 0; j < spc; ++j) {
          const float w = weight(j, r);
          const float2 gv = dv[c * spc + j];
          gk.x = fmaf(w, gv.x, gk.x);
          gk.y = fmaf(w, gv.y, gk.y);
        }
        if (r == 0) {
          const int cp = c == 0 ? ncurve - 1 : c - 1;
          for (int j = 0; j < spc; ++j) {
            const float w = weight(j, 3);
            const float2 gv = dv[cp * spc + j];
            gk.x = fmaf(w, gv.x, gk.x);
            gk.y = fmaf(w, gv.y, gk.y);
          }
        }
      }
      d.dctrl[c0 + k] = gk;
      if (mode == 1) {
        float2 p = d.ctrl[c0 + k], m = d.ctrl_m[c0 + k], v = d.ctrl_v[c0 + k];
        m.x = d.b1 * m.x + (1.0f - d.b1) * gk.x;
        m.y = d.b1 * m.y + (1.0f - d.b1) * gk.y;
        v.x = d.b2 * v.x + (1.0f - d.b2) * gk.x * gk.x;
        v.y = d.b2 * v.y + (1.0f - d.b2) * gk.y * gk.y;
        p.x -= step_size * m.x / (sqrtf(v.x) / bc2s + d.eps);
        p.y -= step_size * m.y / (sqrtf(v.y) / bc2s + d.eps);
        d.ctrl[c0 + k] = p;
        d.ctrl_m[c0 + k] = m;
        d.ctrl_v[c0 + k] = v;
      }
    }
    if (!staged) {
      __syncthreads();  // every read of dv is done
      for (int i = threadIdx.x; i < nv; i += kCtrlThreads) d.dv[v0 + i] = make_float2(0.0f, 0.0f);
    }
    if (mode == 0) return;
    __syncthreads();  // the new points are visible to the block
  }
  // the flattening (the same sampling as the host's at create time)
  for (int i = threadIdx.x; i < nv; i += kCtrlThreads) {
    if (!cubic) {
      d.vloc[v0 + i] = d.ctrl[c0 + i];
      continue;
    }
    const int c = i / spc, j = i % spc;
    float x = 0.0f, y = 0.0f;
    for (int r = 0; r < 4; ++r) {
      const float2 p = d.ctrl[c0 + (3 * c + r) % np];
      const float w = weight(j, r);
      x = fmaf(w, p.x, x);
      y = fmaf(w, p.y, y);
    }
    d.vloc[v0 + i] = make_float2(x, y);
  }
  // bin radius: the largest |point| (the curve stays in the convex hull of its control points;
  // the tile rectangle adds a pixel of slack beyond it)
  float rmax = 0.0f;
  for (int k = threadIdx.x; k < np; k += kCtrlThreads) {
    const float2 p = d.ctrl[c0 + k];
    rmax = fmaxf(rmax, sqrtf(fmaf(p.x, p.x, p.y * p.y)));
  }
  for (int o = 16; o; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0) s_r[threadIdx.x >> 5] = rmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kCtrlThreads / 32; ++w) rmax = fmaxf(rmax, s_r[w]);
    d.elem_rbin[g] = rmax;
  }
}

cudaError_t launch_ctrl_step(const Dev& d, cudaStream_t s, int mode) {
  if (d.n_elems <= 0) return cudaSuccess;
  return klaunch(d.pdl, k_ctrl_step, d.n_elems, kCtrlThreads, 0, s, d, mode);
}

}  // namespace collage
