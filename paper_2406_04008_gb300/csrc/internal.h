// Internal device-side layout of libcollage (not part of the C ABI).
//
// HBM layout, all problems of a handle concatenated:
//   per element g (SoA):   prob, vertex offset, closed flag, stroke half-width, bin radius,
//                          params q / Adam m, v (float4), world translation in pixels (hi, lo),
//                          outline box, tile rectangle, gradient dq
//   per flattened vertex:  local position (unit coords), per-iteration segment record relative to
//                          the element translation in pixels (float, rounded from double)
//   per (tile, element) pair, capacity `cap`: element of each pair in emission order and in
//                          element order, deterministic gradient partials, and per pixel of the
//                          tile the signed distance + closest segment saved by the forward pass
//   per pixel (level):     container coverage, Ihat, prod(1 - tau c^pad), uniform-loss scratch
//   per tile:              counting-sort count, [begin, end) into the pairs, loss partials
#pragma once
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

namespace collage {

constexpr int kMaxDil = 8;
constexpr int kCtlWords = 24;           // device control words (status first, see Dev)
constexpr int kChunkPx = 64;            // side, in pixels, of the emission's chunks of an element
constexpr int kHeavyChunk = 1024;       // segments x tiles above which a chunk is taken first
constexpr int kStatusOverflow = 1;      // device status bits
constexpr int kStatusBadParam = 2;
constexpr int kStatusInternal = 4;      // an internal bounds check failed (a bug)
constexpr int kStatusTileCap = 8;       // a tile's pair list outgrew its capacity (regrown, re-run)
constexpr int kStatusNoBins = kStatusOverflow | kStatusTileCap;  // the bins of the iteration are void
constexpr int kStatusVoid = kStatusNoBins | kStatusBadParam;      // the iteration is void

// Class of a (tile, element) pair.  A pair is near when some segment of the outline lies within
// the coverage margin (rho + pad + stroke half-width) of some pixel centre of the tile; otherwise
// the coverage and the padded coverage are the same saturated value (0 or 1) on every pixel of
// the tile and the pair carries no gradient.
constexpr uint8_t kPairOut = 0;   // not near, outside the outline: c = c^pad = 0
constexpr uint8_t kPairIn = 1;    // not near, inside: c = c^pad = 1
constexpr uint8_t kPairNear = 2;  // per-pixel signed distances (the distance kernel)

struct LossParams {
  float alpha, beta, gamma, delta;
  int force_kind;               // 0: downward potential 1 - y; 1: |p - (fx, fy)|
  float fx, fy;
  float tau, w_in, w_out;
  int n_dil;
  float dil_w[kMaxDil];
  float pad_px, rho_px;
};

struct Dev {
  // ---- problem (fixed at create) ----
  int n_elems, n_probs;
  int max_segs;                 // the most segments of any element
  const int* elem_prob;
  const int* elem_voff;         // [n+1]
  const uint8_t* elem_closed;
  const float* elem_hw;         // unit coords
  float* elem_rbin;             // bin radius (largest |control point|), float
  float2* vloc;                 // flattened local vertices, unit coords (rewritten by
                                //   k_ctrl_step when the outlines are fitted)
  const int* prob_elem_base;    // [P+1]
  const double* ring_pts;       // container rings, unit coords (double)
  const int* ring_off;          // [total rings + 1]
  const int* prob_ring_base;    // [P+1] into ring_off
  // ---- level ----
  const int* prob_res;          // [P]
  const int* prob_ntx;          // [P] tiles per side
  const int* prob_tile_base;    // [P+1]
  const long long* prob_pix_base;  // [P+1]
  const int* prob_dtile_base;   // [P+1] dilation tiles
  int total_tiles, total_dtiles;
  long long total_pix;
  int tile;                     // raster tile side
  int emit_threads;             // threads per block of the emission / distance kernel (128, 256)
  int chunk_tiles;              // side of the emission's chunks, in tiles (<= kChunkPx / tile)
  int n_sort_passes;
  // ---- params / optimiser ----
  float4* q;
  float4* m;
  float4* v;
  const float4* q_in;           // [n] params the transform takes in place of q (the host-buffer
                                //   step's mapped input), or null
  const uchar4* trainable;      // may be null
  float lr, b1, b2, eps, s_min, s_max;
  // ---- per iteration ----
  float4* segA;                 // [V] segment k: start (px, relative to the translation), direction
  float2* segB;                 // [V] segment k: end point y, 1 / |direction|^2
  float* segS;                  // [V] segment k: dx/dy of its direction (0 if horizontal)
  float4* tpx;                  // [n] translation in px: (hi.x, hi.y, lo.x, lo.y)
  float4* bbox;                 // [n] outline box relative to the translation, grown by the margin
  int4* rect;                   // [n] tile rectangle (tx0, ty0, tx1, ty1), empty if tx1 < tx0
  int* elem_pbase;              // [n] first pair slot of each element: its tile rectangle's pairs
                                //   take consecutive slots, row-major (the transform allocates them)
  int* pair_need;               // [1] pair slots allocated by this iteration's transform
  int* total_pairs;             // [1] pairs of the last binning (copied from pair_need)
  int cap;                      // pair capacity
  int* tile_n;                  // [total_tiles] pairs registered in each tile's list by the
                                //   emission (the composite zeroes it)
  int* tile_m;                  // [total_tiles] pairs of each tile (the composite's count, kept)
  int* tile_list;               // [total_tiles * tile_cap] pair slots of each tile, emission order
  int* tile_sorted;             // [total_tiles * tile_cap] each tile's elements in increasing order
  int* tile_sorted_slot;        //   and their pair slots (written by the composite)
  int tile_cap;                 // pair-list capacity of a tile
  int* tile_max;                // [1] pairs of the fullest tile list of the iteration (the
                                //   composite's maximum; the emission's block 0 zeroes it)
  int* pair_elem;               // [cap] element of each pair slot (tile ranges, emission order)
  uint8_t* pair_cls;            // [cap] kPairOut / kPairIn / kPairNear, set by the emission
  int4* near_list;              // [list_cap] the emission's work list: (element, chunk origin tile
                                //   column | row << 16, problem, 0), one per kChunkPx-square chunk of
                                //   every element's tile rectangle, appended by the transform: heavy
                                //   ones from the front, light ones from the back
  int list_cap;                 // entries near_list holds
  int* chunk_count;             // [2] heavy and light chunks appended by the transform (the
                                //   composite's block 0 zeroes them)
  int4* live_list;              // [cap] pairs with some non-saturated pixel: (slot, element, tile
                                //   column | row << 16, problem), the adjoint's work list (order
                                //   depends on atomics)
  float2* saved;                // [cap * tile*tile] (sd px, closest segment as int bits)
  float* covc;                  // [pix] container coverage
  float* img_I;                 // [pix] Ihat = prod(1 - c)
  float* img_Pt;                // [pix] +-prod(1 - tau c^pad), negative where A_tau > tau
  float* gOu;                   // [pix] dL_u/dO
  uint32_t* dil_g;              // [pix] the adjoint's staged word: round(M_C (1 - O) 2^Q) in bits
                                // 0..23, bit 24 + k set where B_k < 1 (Q of the kernel count)
  float4* lossA;                // [total_tiles] (sum W(I-Ic)^2, sum relu(A-tau), sum O(1-y), 0)
  float* lossU;                 // [total_dtiles] weighted uniform-loss partial
  uint8_t* dtile_flags;         // [total_dtiles] container coverage on the tile / its halo (or null)
  int* dtile_list;              // [2 total_dtiles] the tiles with kFlagOwn from 0, with kFlagHalo
                                //   from total_dtiles, in no particular order (or null: all tiles)
  int* dtile_n;                 // [2] lengths of the two lists
  float4* dq;                   // [n] gradient
  float4* partial;              // [cap] deterministic gradient partials, at emit position
  float* loss_terms;            // [P*5]
  int* status;                  // [1]
  int* step;                    // [1] Adam step count (the loss assembly advances it)
  int* pending;                 // [1] 1: the Adam step `step` is computed (dq) but not yet applied
  int* sched_base;              // [1] Adam step count when the running schedule graph began
  int* work;                    // [8] per-iteration counters: [0] chunks taken by the emission's
                                //   blocks beyond the first (the composite's block 0 zeroes it), [1] entries of live_list and
                                //   [3] blocks of the last gradient kernel that have finished
                                //   (zeroed by the transform), [5] blocks of the Adam flush that
                                //   have finished (its last block zeroes it), [2, 4, 6, 7] spare
  unsigned long long* paths;    // [4] cumulative counts of the rarely taken kernel paths (since
                                //   create): [0] pixel rows of a near pair whose crossings
                                //   overflow the per-row list (winding over every segment),
                                //   [1] emission chunks of outlines with more segments than
                                //   are staged in shared memory,
                                //   [2] tiles listing more than 32 pairs (ranked in global
                                //   memory), [3] container ring chunks after a ring's first
  LossParams L;
  int deterministic;
  int pdl;                      // launch the iteration's kernels with programmatic serialisation
  // ---- outline fitting (fit_controls): the points of each element are the parameters ----
  int fit;                      // 1: the adjoint accumulates dv and k_ctrl_step runs Adam on ctrl
  int spc;                      // segments per cubic
  const int* elem_coff;         // [n+1] CSR offsets of each element's points in ctrl
  const uint8_t* elem_cubic;    // [n] 1: closed cubic path (points are control points)
  float2* ctrl;                 // [C] points, element-local unit coordinates
  float2* ctrl_m;               // [C] Adam moments
  float2* ctrl_v;
  float2* dctrl;                // [C] dL/d(points) of the last backward pass
  float2* dv;                   // [V] dL/d(flattened vertex), element-local unit coordinates
};

// ---- the checked build (-DCOLLAGE_CHECKED, libcollage_checked.so) ----
// in_bounds(d, ok): a failed index check latches kStatusInternal (the next host call that reads
// the status word returns COLLAGE_ERR_STATE) and the caller skips the guarded access, so nothing
// is read or written past a bound and nothing traps; the checked build also prints the first
// failures' source lines.  In the regular build it is the constant true and compiles away.
#ifdef COLLAGE_CHECKED
static __device__ int g_bounds_reports = 0;
__device__ __forceinline__ bool in_bounds_at(const Dev& d, bool ok, int line, const char* file) {
  if (!ok) {
    atomicOr(d.status, kStatusInternal);
    if (atomicAdd(&g_bounds_reports, 1) < 8) printf("collage: bounds check failed at %s:%d\n", file, line);
  }
  return ok;
}
#define in_bounds(d, ok) in_bounds_at((d), (ok), __LINE__, __FILE__)
#else
__device__ __forceinline__ bool in_bounds(const Dev& d, bool ok) {
  (void)d;
  (void)ok;
  return true;
}
#endif

// Adam (bias-corrected, the update torch.optim.Adam performs; it stands in for the plain descent
// step of Eq. 4) of element g at step t >= 1 with gradient gr, then the clamp of s.
// An iteration's step is applied lazily: the loss assembly marks it pending, and the next
// iteration's transform kernel (one block per element, which reads the params first anyway)
// applies it before forming the geometry; API calls that read or replace params flush it.
__device__ __forceinline__ void adam_apply(const Dev& d, int t, float4 gr, uchar4 tr, float4& q, float4& m,
                                           float4& v) {
  const float bc1 = 1.0f - powf(d.b1, (float)t), bc2 = 1.0f - powf(d.b2, (float)t);
  const float step_size = d.lr / bc1, bc2s = sqrtf(bc2);
  float* qp = &q.x;
  float* mp = &m.x;
  float* vp = &v.x;
  const float gg[4] = {gr.x, gr.y, gr.z, gr.w};
  const unsigned char tt[4] = {tr.x, tr.y, tr.z, tr.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!tt[k]) continue;
    mp[k] = d.b1 * mp[k] + (1.0f - d.b1) * gg[k];
    vp[k] = d.b2 * vp[k] + (1.0f - d.b2) * gg[k] * gg[k];
    const float denom = sqrtf(vp[k]) / bc2s + d.eps;
    qp[k] -= step_size * mp[k] / denom;
  }
  q.w = fminf(fmaxf(q.w, d.s_min), d.s_max);
}
__device__ __forceinline__ void adam_update(const Dev& d, int g, int t, float4 gr) {
  float4 q = d.q[g], m = d.m[g], v = d.v[g];
  const uchar4 tr = d.trainable ? d.trainable[g] : make_uchar4(1, 1, 1, 1);
  adam_apply(d, t, gr, tr, q, m, v);
  d.q[g] = q;
  d.m[g] = m;
  d.v[g] = v;
}

// Potential of the force term at the pixel centre (px, py), unit coordinates.
__device__ __forceinline__ float force_potential(const LossParams& L, float px, float py) {
  if (L.force_kind == 1) return hypotf(px - L.fx, py - L.fy);
  return 1.0f - py;
}

// ---- programmatic dependent launch ----
// With Dev::pdl set, the kernels of an iteration are launched with programmatic stream
// serialisation: a kernel may be scheduled while its predecessor on the stream still runs.  Every
// such kernel starts with pdl_enter(): griddepcontrol.wait returns once the predecessor grid has
// completed and its memory operations are visible (before any global access or early return, so
// completion stays transitive along the chain), then launch_dependents lets the successor be
// scheduled.  Launched without the attribute, both instructions are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t klaunch(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                           cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// The last block of the kernel that completes an iteration's gradient marks the iteration's Adam
// step pending (applied by the next transform) and advances the step count, unless the iteration
// overflowed or met non-finite params.  Every block calls this once, after its last write to the
// gradient; the counter work[3] is zeroed by the tile scan of each iteration.
__device__ __forceinline__ void mark_step_if_last(const Dev& d) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's gradient writes are visible before it is counted
    if (atomicAdd(&d.work[3], 1) == (int)gridDim.x - 1 && !(atomicAdd(d.status, 0) & kStatusVoid)) {
      __threadfence();
      *d.step += 1;
      *d.pending = 1;
    }
  }
}

// ---- launchers (each enqueues on `s`, returns the launch error) ----
cudaError_t launch_transform(const Dev& d, cudaStream_t s, bool zero_grad);
cudaError_t launch_container(const Dev& d, cudaStream_t s);
// part 1: pair emission, classification and per-pixel signed distances (per element chunk);
// part 2: per-tile composite and loss partials; 3: both
cudaError_t launch_raster_fwd(const Dev& d, cudaStream_t s, int pair_grid, int tile_grid,
                              float* out_bw, float* out_tau, int part = 3);
cudaError_t prepare_dilate(int n_dil);  // sets dynamic shared memory limits (not capturable)
cudaError_t launch_dilate(const Dev& d, cudaStream_t s, bool backward);
cudaError_t launch_dtile_flags(const Dev& d, cudaStream_t s);  // once per level, after the container
// mark_step: the kernel's last block marks the iteration's Adam step (step mode)
cudaError_t launch_raster_bwd(const Dev& d, cudaStream_t s, int pair_grid, bool mark_step);
cudaError_t launch_grad_reduce(const Dev& d, cudaStream_t s, bool mark_step);
// applies a pending Adam step to all elements and clears the flag (before params are read)
cudaError_t launch_adam_flush(const Dev& d, cudaStream_t s, float* out = nullptr);
// outline fitting, one block per element: mode 0 maps dv to dctrl (and clears dv); mode 1 also
// takes an Adam step on ctrl at step *d.step and flattens again (vertices and bin radii); mode 2
// only flattens
cudaError_t launch_ctrl_step(const Dev& d, cudaStream_t s, int mode);
// skeleton-based initialisation: distance transform, medial axis, greedy placement into d.q
cudaError_t launch_mat_init(const Dev& d, cudaStream_t s, int max_res, int* gcol, unsigned* d2,
                            int* cand, int* n_cand, float* clear, int* order, int* axis_out,
                            float* width_out);
cudaError_t launch_loss(const Dev& d, cudaStream_t s);
// the captured level schedule: records the step count at the start of a run; sets a level's loop
// condition (1 while fewer than `target` iterations of the run are done and nothing latched)
cudaError_t launch_sched_begin(const Dev& d, cudaStream_t s);
cudaError_t launch_sched_cond(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle cond, int target);
cudaError_t launch_copy_grad(const Dev& d, cudaStream_t s, float* out);
// Resident blocks per SM of the raster kernels, the pairs one adjoint block and the tiles one
// composite block take at once (the forward distance kernel takes one pair per block).
struct RasterOcc {
  int fwd_per_sm, bwd_per_sm, tile_per_sm, bwd_pairs_per_block, tiles_per_block;
};
void raster_occupancy(int tile, int emit_threads, RasterOcc* o);
// quality metrics after a render pass: counts [4 * n_probs] and squared-distance sums [n_probs]
cudaError_t launch_metrics(const Dev& d, cudaStream_t s, uint8_t* obj, int* gcol,
                           unsigned long long* cnt, unsigned long long* sums, int max_res);

}  // namespace collage
