// Host side of libcollage: argument validation, flattening of cubic paths, device buffers, the
// per-level setup (container raster, bin capacity), the iteration sequence, CUDA-graph capture,
// stage timing, the tile autotuner and the C ABI of include/collage.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "collage.h"
#include "internal.h"

#ifdef COLLAGE_CHECKED
#include <nvtx3/nvToolsExt.h>
#endif

using namespace collage;

namespace {

thread_local std::string g_create_error;

enum Mode { kRender = 0, kLossBwd = 1, kStep = 2 };

}  // namespace

struct collage_s {
  collage_options opt{};
  int P = 0, N = 0, V = 0;
  // host copies of the problem
  std::vector<int> elem_prob, elem_voff, prob_elem_base, prob_grid, ring_off, prob_ring_base;
  std::vector<uint8_t> elem_closed;
  std::vector<float> elem_hw, elem_rbin;
  std::vector<float2> vloc;
  std::vector<float2> ctrl;        // the problems' points (cubic control points, polygon and
  std::vector<int> elem_coff;      //   polyline vertices), CSR by element
  std::vector<uint8_t> elem_cubic;
  std::vector<double> ring_pts;
  bool has_trainable = false;
  // level state
  int level = -1;
  std::vector<int> res, ntx, tile_base, dtile_base;  // host copies of the current level's tables
  std::vector<long long> pix_base;
  // every level's tables for the raster tile lv_tile: host copies and device arrays
  struct LevelTab {
    std::vector<int> res, ntx, tile_base, dtile_base;
    std::vector<long long> pix_base;
    int total_tiles = 0, total_dtiles = 0;
    long long total_pix = 0;
    int* d_res = nullptr;
    int* d_ntx = nullptr;
    int* d_tile_base = nullptr;
    int* d_dtile_base = nullptr;
    long long* d_pix_base = nullptr;
  };
  std::vector<LevelTab> lv;
  int lv_tile = 0;
  int pair_grid = 0;  // grid of the emission / distance kernel
  int bwd_grid = 0;   // grid of the per-pair adjoint
  int tile_grid = 0;  // grid of the per-tile composite
  int sms = 1;
  // launch configuration (the autotuner's choice): persistent grids are these multiples of the SM
  // count x resident blocks per SM
  float fwd_mult = 1.0f, bwd_mult = 1.0f, comp_mult = 1.0f;
  collage_tuning tuning{};
  // device memory
  Dev d{};
  size_t pix_cap = 0, tile_cap = 0, dtile_cap = 0, pair_cap = 0, saved_tile = 0;
  std::vector<void*> list_bufs;  // per-tile pair lists: tile_cap tiles x d.tile_cap entries
  int* ctl = nullptr;        // device: status, step, total_pairs, pending, 8 work counters,
                             //   schedule base step, 2 chunk counts, pairs allocated, 1 spare,
                             //   fullest tile list, 6 spare
  int* h_ctl = nullptr;      // pinned mirror
  float* d_stage = nullptr;  // device: params, loss terms and control words gathered for one copy
  float* h_stage = nullptr;  // pinned: their host copy ([4n | 5 n_probs | 4], see k_adam_flush)
  float* h_stage_dev = nullptr;  // h_stage mapped into the device's address space (or null): the
                                 // gathering kernel then writes the host copy itself
  float* h_in = nullptr;         // pinned, mapped: params in for the host-buffer step ([4n])
  float4* h_in_dev = nullptr;    // h_in in the device's address space (or null: no host graph)
  bool ctl_current = false;  // h_ctl[1] (step count) and h_ctl[3] (pending) are the device's:
                             // no step was enqueued since the last read
  cudaStream_t cap_stream = nullptr;
  cudaStream_t aux_stream = nullptr;  // side branch of an iteration (the loss assembly)
  cudaStream_t body_stream = nullptr;  // captures the loop bodies of the schedule graph
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t graph = nullptr;  // one iteration at the current level
  cudaGraphExec_t host_graph = nullptr;  // one iteration taking its params from h_in, then the
                                         // gathering kernel writing h_stage (collage_step_host)
  cudaGraphExec_t sched = nullptr;  // the schedule from level sched_start to the last
  int sched_start = -1;
  // quality-metric scratch (allocated by collage_metrics)
  uint8_t* met_obj = nullptr;
  int* met_gcol = nullptr;
  unsigned long long* met_cnt = nullptr;  // [5 * P]: 4 counts, then the distance sums
  // skeleton-based initialisation scratch (allocated by collage_mat_init)
  unsigned char* mat_buf = nullptr;
  size_t mat_bytes = 0;
  size_t met_pix = 0;
  std::string err;
  std::vector<void*> owned;      // fixed-size allocations
  std::vector<void*> level_bufs; // per-pixel / per-tile buffers, regrown with the level size
  std::vector<void*> pair_bufs;  // per-pair buffers, regrown with the bin capacity

  ~collage_s();
};

namespace {

collage_status fail(collage_t h, collage_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return st;
}

collage_status cuda_fail(collage_t h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(h, e == cudaErrorMemoryAllocation ? COLLAGE_ERR_OOM : COLLAGE_ERR_CUDA, m);
}

#define CK(h, expr)                                       \
  do {                                                    \
    cudaError_t e_ = (expr);                              \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #expr); \
  } while (0)

template <class T>
cudaError_t dmalloc(std::vector<void*>& list, T*& p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(n, 1));
  if (e != cudaSuccess) return e;
  list.push_back(q);
  p = static_cast<T*>(q);
  return cudaSuccess;
}

template <class T>
cudaError_t upload(std::vector<void*>& list, T*& p, const std::vector<T>& v) {
  cudaError_t e = dmalloc(list, p, v.size());
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  return e;
}

void free_list(std::vector<void*>& list) {
  for (void* p : list) cudaFree(p);
  list.clear();
}

bool is_finite_f(float x) { return std::isfinite(x); }

// The one-iteration graph holds the current level's tables; the schedule graph holds every level's
// but the pair buffers, tile size and grids of its capture.
void drop_iter_graph(collage_t h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  if (h->host_graph) cudaGraphExecDestroy(h->host_graph);
  h->host_graph = nullptr;
}

void drop_graph(collage_t h) {
  drop_iter_graph(h);
  if (h->sched) cudaGraphExecDestroy(h->sched);
  h->sched = nullptr;
  h->sched_start = -1;
}

}  // namespace

collage_s::~collage_s() {
  if (graph) cudaGraphExecDestroy(graph);
  if (host_graph) cudaGraphExecDestroy(host_graph);
  if (h_in) cudaFreeHost(h_in);
  if (sched) cudaGraphExecDestroy(sched);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  if (body_stream) cudaStreamDestroy(body_stream);
  if (aux_stream) cudaStreamDestroy(aux_stream);
  if (met_obj) cudaFree(met_obj);
  if (met_gcol) cudaFree(met_gcol);
  if (met_cnt) cudaFree(met_cnt);
  if (mat_buf) cudaFree(mat_buf);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (h_ctl) cudaFreeHost(h_ctl);
  if (h_stage) cudaFreeHost(h_stage);
  free_list(pair_bufs);
  free_list(list_bufs);
  free_list(level_bufs);
  free_list(owned);
}

// --------------------------------------------------------------------------------------------
// Options and validation
// --------------------------------------------------------------------------------------------
extern "C" void collage_default_options(collage_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->alpha = 3e3f;
  o->beta = 8e4f;
  o->gamma = 5e-4f;
  o->delta_down = 0.0f;
  o->tau = 0.5f;
  o->w_in = 1.0f;
  o->w_out = 100.0f;
  o->n_dilations = 4;
  for (int k = 0; k < 8; ++k) o->dil_weight[k] = (float)(k + 1);
  o->pad_px = 0.0f;
  o->rho_px = 1.0f;
  o->segs_per_cubic = 16;
  o->n_levels = 1;
  o->level_res[0] = 1024;
  o->level_iters[0] = 50;
  o->lr = 1e-2f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  o->s_min = 0.05f;
  o->s_max = 20.0f;
  o->deterministic = 0;
  o->tile = 16;
  o->persistent = 1;
  o->use_graphs = 1;
  o->overlap_launches = 1;
  o->force_kind = 0;
  o->force_x = 0.5f;
  o->force_y = 0.5f;
}

static std::string check_options(const collage_options& o) {
  if (o.n_levels < 1 || o.n_levels > 8) return "n_levels must be in 1..8";
  for (int l = 0; l < o.n_levels; ++l) {
    if (o.level_res[l] < 1) return "level_res[" + std::to_string(l) + "] must be >= 1";
    if (o.level_iters[l] < 0) return "level_iters[" + std::to_string(l) + "] must be >= 0";
  }
  if (!(o.tile == 0 || o.tile == 8 || o.tile == 16)) return "tile must be 0, 8 or 16";
  if (o.fit_controls != 0 && o.fit_controls != 1) return "fit_controls must be 0 or 1";
  if (o.n_dilations < 0 || o.n_dilations > 8) return "n_dilations must be in 0..8";
  const float f[] = {o.alpha, o.beta, o.gamma, o.delta_down, o.w_in, o.w_out, o.lr, o.eps};
  for (float x : f)
    if (!is_finite_f(x)) return "loss weights, penalties, lr and eps must be finite";
  for (int k = 0; k < o.n_dilations; ++k)
    if (!is_finite_f(o.dil_weight[k])) return "dil_weight must be finite";
  if (!(o.rho_px > 0.0f) || !is_finite_f(o.rho_px)) return "rho_px must be > 0";
  if (!(o.pad_px >= 0.0f) || !is_finite_f(o.pad_px)) return "pad_px must be >= 0";
  if (!(o.tau > 0.0f && o.tau < 1.0f)) return "tau must be in (0, 1)";
  if (o.segs_per_cubic < 1 || o.segs_per_cubic > 4096) return "segs_per_cubic must be in 1..4096";
  if (!(o.beta1 >= 0.0f && o.beta1 < 1.0f) || !(o.beta2 >= 0.0f && o.beta2 < 1.0f)) return "Adam betas must be in [0, 1)";
  if (!(o.s_min > 0.0f) || !(o.s_max >= o.s_min) || !is_finite_f(o.s_max)) return "need 0 < s_min <= s_max";
  if (o.force_kind != 0 && o.force_kind != 1) return "force_kind must be 0 or 1";
  if (!is_finite_f(o.force_x) || !is_finite_f(o.force_y)) return "force_x and force_y must be finite";
  return "";
}

static std::string check_problem(const collage_problem& p, int idx, const collage_options& o) {
  const std::string at = "problem " + std::to_string(idx) + ": ";
  if (p.n_elems < 1) return at + "n_elems must be >= 1";
  if (!p.kind || !p.pt_off || !p.pts || !p.params0) return at + "kind, pt_off, pts and params0 are required";
  if (p.pt_off[0] != 0) return at + "pt_off[0] must be 0";
  for (int e = 0; e < p.n_elems; ++e) {
    const int np = p.pt_off[e + 1] - p.pt_off[e];
    const std::string ae = at + "element " + std::to_string(e) + ": ";
    switch (p.kind[e]) {
      case COLLAGE_CUBIC_PATH:
        if (np < 3 || np % 3) return ae + "a cubic path needs 3N >= 3 control points";
        break;
      case COLLAGE_POLYGON:
        if (np < 3) return ae + "a polygon needs >= 3 points";
        break;
      case COLLAGE_POLYLINE:
        if (np < 2) return ae + "a polyline needs >= 2 points";
        if (p.stroke_hw && !(p.stroke_hw[e] >= 0.0f && is_finite_f(p.stroke_hw[e]))) return ae + "stroke_hw must be finite and >= 0";
        break;
      default:
        return ae + "unknown kind";
    }
    for (int k = 2 * p.pt_off[e]; k < 2 * p.pt_off[e + 1]; ++k)
      if (!is_finite_f(p.pts[k])) return ae + "points must be finite";
    const float* q = p.params0 + 4 * e;
    for (int k = 0; k < 4; ++k)
      if (!is_finite_f(q[k])) return ae + "params must be finite";
    if (!(q[3] > 0.0f)) return ae + "scale s must be > 0";
  }
  if (p.n_rings < 1 || !p.ring_off || !p.ring_pts) return at + "a container needs >= 1 ring";
  if (p.ring_off[0] != 0) return at + "ring_off[0] must be 0";
  for (int r = 0; r < p.n_rings; ++r) {
    if (p.ring_off[r + 1] - p.ring_off[r] < 3) return at + "each container ring needs >= 3 points";
    for (int k = 2 * p.ring_off[r]; k < 2 * p.ring_off[r + 1]; ++k)
      if (!is_finite_f(p.ring_pts[k])) return at + "container points must be finite";
  }
  if (p.grid < 0) return at + "grid must be >= 0";
  const long long g = p.grid ? p.grid : o.level_res[o.n_levels - 1];
  const long long last = o.level_res[o.n_levels - 1];
  for (int l = 0; l < o.n_levels; ++l) {
    if ((g * o.level_res[l]) % last) return at + "grid * level_res[l] must be divisible by level_res[last]";
    if (g * o.level_res[l] / last < 1) return at + "a level resolution rounds to 0";
    if (g * o.level_res[l] / last > 32768) return at + "a level resolution exceeds 32768";
  }
  return "";
}

// --------------------------------------------------------------------------------------------
// Flattening (Sec. 3 "Vector Representation"): curve k of a closed cubic path uses control points
// 3k, 3k+1, 3k+2, 3k+3 (mod 3N), sampled at t = j / segs (j = 0..segs-1), Bernstein form, double.
// --------------------------------------------------------------------------------------------
static void flatten(const collage_problem& p, int e, int spc, std::vector<float2>& out, float& rbin) {
  const float* pts = p.pts + 2 * p.pt_off[e];
  const int np = p.pt_off[e + 1] - p.pt_off[e];
  double rmax = 0.0;
  for (int k = 0; k < np; ++k) {
    const double x = pts[2 * k], y = pts[2 * k + 1];
    rmax = std::max(rmax, std::sqrt(x * x + y * y));
  }
  rbin = (float)rmax;
  if (p.kind[e] != COLLAGE_CUBIC_PATH) {
    for (int k = 0; k < np; ++k) out.push_back(make_float2(pts[2 * k], pts[2 * k + 1]));
    return;
  }
  for (int k = 0; k < np / 3; ++k) {
    const float* c[4];
    for (int i = 0; i < 4; ++i) c[i] = pts + 2 * ((3 * k + i) % np);
    for (int j = 0; j < spc; ++j) {
      const double t = (double)j / spc, u = 1.0 - t;
      const double b[4] = {u * u * u, 3.0 * u * u * t, 3.0 * u * t * t, t * t * t};
      double x = 0.0, y = 0.0;
      for (int i = 0; i < 4; ++i) {
        x += b[i] * c[i][0];
        y += b[i] * c[i][1];
      }
      out.push_back(make_float2((float)x, (float)y));
    }
  }
}

// --------------------------------------------------------------------------------------------
// Level setup
// --------------------------------------------------------------------------------------------
// Persistent grids: resident blocks per SM times the SM count; plain grids: one block per work
// item (pairs up to the capacity, every tile).
static void set_grids(collage_t h) {
  RasterOcc o{};
  raster_occupancy(h->d.tile, h->d.emit_threads, &o);
  auto scaled = [&](int per_sm, float mult) { return std::max(1, (int)std::lround(h->sms * per_sm * mult)); };
  if (h->opt.persistent) {
    h->pair_grid = scaled(o.fwd_per_sm, h->fwd_mult);
    h->bwd_grid = scaled(o.bwd_per_sm, h->bwd_mult);
    h->tile_grid = std::min((h->d.total_tiles + o.tiles_per_block - 1) / o.tiles_per_block,
                            scaled(o.tile_per_sm, h->comp_mult));
  } else {
    h->pair_grid = std::max(h->d.cap, 1);
    h->bwd_grid = std::max((h->d.cap + o.bwd_pairs_per_block - 1) / o.bwd_pairs_per_block, 1);
    h->tile_grid = (h->d.total_tiles + o.tiles_per_block - 1) / o.tiles_per_block;
  }
}

static collage_status ensure_pairs(collage_t h, size_t cap) {
  const size_t tt = (size_t)h->d.tile * h->d.tile;
  if (cap <= h->pair_cap && tt == h->saved_tile) return COLLAGE_OK;
  drop_graph(h);
  CK(h, cudaDeviceSynchronize());
  free_list(h->pair_bufs);
  h->pair_cap = 0;
  Dev& d = h->d;
  CK(h, dmalloc(h->pair_bufs, d.pair_elem, cap));
  CK(h, dmalloc(h->pair_bufs, d.live_list, cap));
  CK(h, dmalloc(h->pair_bufs, d.near_list, cap));
  CK(h, dmalloc(h->pair_bufs, d.pair_cls, cap));
  CK(h, dmalloc(h->pair_bufs, d.partial, cap));
  CK(h, dmalloc(h->pair_bufs, d.saved, cap * tt));
  h->pair_cap = cap;
  h->saved_tile = tt;
  d.cap = (int)std::min<size_t>(cap, 0x7fffffff);
  d.list_cap = d.cap;
  set_grids(h);
  return COLLAGE_OK;
}

// floats of the gathered output: params, loss terms, control words
static size_t stage_floats(const collage_s* h) { return 4 * (size_t)h->N + 5 * (size_t)h->P + kCtlWords; }

static collage_status read_ctl(collage_t h, cudaStream_t s) {
  CK(h, cudaMemcpyAsync(h->h_ctl, h->ctl, kCtlWords * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  h->ctl_current = true;
  return COLLAGE_OK;
}

// Per-tile pair lists of capacity `per_tile` for the largest level's tiles.
static collage_status ensure_tile_lists(collage_t h, int per_tile) {
  drop_graph(h);
  CK(h, cudaDeviceSynchronize());
  free_list(h->list_bufs);
  Dev& d = h->d;
  const size_t n = h->tile_cap * (size_t)per_tile;
  CK(h, dmalloc(h->list_bufs, d.tile_list, n));
  CK(h, dmalloc(h->list_bufs, d.tile_sorted, n));
  CK(h, dmalloc(h->list_bufs, d.tile_sorted_slot, n));
  d.tile_cap = per_tile;
  return COLLAGE_OK;
}

// Per-pixel, per-tile and per-dilation-tile buffers for the largest level (regrown if needed).
static collage_status ensure_level_bufs(collage_t h, size_t np, size_t nt, size_t nd) {
  if (np <= h->pix_cap && nt <= h->tile_cap && nd <= h->dtile_cap) return COLLAGE_OK;
  drop_graph(h);
  CK(h, cudaDeviceSynchronize());
  free_list(h->level_bufs);
  h->pix_cap = h->tile_cap = h->dtile_cap = 0;
  Dev& d = h->d;
  CK(h, dmalloc(h->level_bufs, d.covc, np));
  CK(h, dmalloc(h->level_bufs, d.img_I, np));
  CK(h, dmalloc(h->level_bufs, d.img_Pt, np));
  CK(h, dmalloc(h->level_bufs, d.gOu, np));
  CK(h, dmalloc(h->level_bufs, d.dil_g, np));
  CK(h, dmalloc(h->level_bufs, d.tile_n, nt));
  CK(h, cudaMemset(d.tile_n, 0, sizeof(int) * nt));
  CK(h, dmalloc(h->level_bufs, d.tile_m, nt));
  CK(h, cudaMemset(d.tile_m, 0, sizeof(int) * nt));
  CK(h, dmalloc(h->level_bufs, d.lossA, nt));
  CK(h, dmalloc(h->level_bufs, d.lossU, nd));
  CK(h, dmalloc(h->level_bufs, d.dtile_flags, nd));
  CK(h, dmalloc(h->level_bufs, d.dtile_list, 2 * nd));
  CK(h, dmalloc(h->level_bufs, d.dtile_n, 2));
  h->pix_cap = np;
  h->tile_cap = nt;
  h->dtile_cap = nd;
  return ensure_tile_lists(h, d.tile_cap);
}

// Every level's tables for the current raster tile: per problem the resolution, tiles per side and
// the base offsets of its tiles, dilation tiles and pixels; uploaded once, selected per level.
static collage_status build_levels(collage_t h) {
  const collage_options& o = h->opt;
  const int T = h->d.tile, L = o.n_levels, P = h->P;
  const long long last = o.level_res[L - 1];
  h->lv.resize(L);
  size_t np = 0, nt = 0, nd = 0;
  for (int l = 0; l < L; ++l) {
    collage_s::LevelTab& t = h->lv[l];
    t.res.assign(P, 0);
    t.ntx.assign(P, 0);
    t.tile_base.assign(P + 1, 0);
    t.dtile_base.assign(P + 1, 0);
    t.pix_base.assign(P + 1, 0);
    for (int p = 0; p < P; ++p) {
      const int r = (int)((long long)h->prob_grid[p] * o.level_res[l] / last);
      t.res[p] = r;
      t.ntx[p] = (r + T - 1) / T;
      t.tile_base[p + 1] = t.tile_base[p] + t.ntx[p] * t.ntx[p];
      const int ndt = (r + 31) / 32;
      t.dtile_base[p + 1] = t.dtile_base[p] + ndt * ndt;
      t.pix_base[p + 1] = t.pix_base[p] + (long long)r * r;
    }
    t.total_tiles = t.tile_base[P];
    t.total_dtiles = t.dtile_base[P];
    t.total_pix = t.pix_base[P];
    np = std::max(np, (size_t)t.total_pix);
    nt = std::max(nt, (size_t)t.total_tiles);
    nd = std::max(nd, (size_t)t.total_dtiles);
    if (!t.d_res) {
      CK(h, dmalloc(h->owned, t.d_res, P));
      CK(h, dmalloc(h->owned, t.d_ntx, P));
      CK(h, dmalloc(h->owned, t.d_tile_base, P + 1));
      CK(h, dmalloc(h->owned, t.d_dtile_base, P + 1));
      CK(h, dmalloc(h->owned, t.d_pix_base, P + 1));
    }
    CK(h, cudaMemcpy(t.d_res, t.res.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(t.d_ntx, t.ntx.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(t.d_tile_base, t.tile_base.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(t.d_dtile_base, t.dtile_base.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(t.d_pix_base, t.pix_base.data(), sizeof(long long) * (P + 1), cudaMemcpyHostToDevice));
  }
  drop_graph(h);
  collage_status st = ensure_level_bufs(h, np, nt, nd);
  if (st) return st;
  h->lv_tile = T;
  return COLLAGE_OK;
}

// Points the device view at level `level`'s tables (no device work unless the tile changed).
static collage_status apply_level(collage_t h, int level) {
  if (h->lv_tile != h->d.tile) {
    collage_status st = build_levels(h);
    if (st) return st;
  }
  const collage_s::LevelTab& t = h->lv[level];
  Dev& d = h->d;
  d.prob_res = t.d_res;
  d.prob_ntx = t.d_ntx;
  d.prob_tile_base = t.d_tile_base;
  d.prob_dtile_base = t.d_dtile_base;
  d.prob_pix_base = t.d_pix_base;
  d.total_tiles = t.total_tiles;
  d.total_dtiles = t.total_dtiles;
  d.total_pix = t.total_pix;
  h->res = t.res;
  h->ntx = t.ntx;
  h->tile_base = t.tile_base;
  h->dtile_base = t.dtile_base;
  h->pix_base = t.pix_base;
  return COLLAGE_OK;
}

// The level switch on the device (capturable): the container raster of the level, and the
// distribution term's tile lists with the zeros that the tiles off those lists keep.
static cudaError_t enqueue_level_switch(const Dev& d, cudaStream_t s) {
  cudaError_t e = launch_container(d, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.dtile_n, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.gOu, 0, sizeof(float) * (size_t)d.total_pix, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.dil_g, 0, sizeof(uint32_t) * (size_t)d.total_pix, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.lossU, 0, sizeof(float) * (size_t)d.total_dtiles, s);
  if (e == cudaSuccess) e = launch_dtile_flags(d, s);
  return e;
}

// Pairs that binning the current params at the selected level produces: the transform with an
// unbounded capacity allocates the slots, and their count is read back (synchronises the stream).
// A pending Adam step is applied on the way, as the next iteration would.
static collage_status probe_pairs(collage_t h, cudaStream_t s, size_t* need) {
  Dev& d = h->d;
  Dev probe = d;
  probe.cap = 0x7fffffff;
  probe.list_cap = 0;  // no chunk is listed
  CK(h, launch_transform(probe, s, false));
  CK(h, cudaMemcpyAsync(h->h_ctl + 2, d.pair_need, sizeof(int), cudaMemcpyDeviceToHost, s));
  // the probe allocated slots and counted chunks without an emission: reset both, and the pending
  // Adam step it applied
  CK(h, cudaMemsetAsync(d.pair_need, 0, sizeof(int), s));
  CK(h, cudaMemsetAsync(d.chunk_count, 0, 2 * sizeof(int), s));
  CK(h, cudaMemsetAsync(d.pending, 0, sizeof(int), s));
  CK(h, cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  h->h_ctl[3] = 0;
  h->ctl_current = false;  // h_ctl[1] was not read
  if (h->h_ctl[0] & kStatusBadParam) return fail(h, COLLAGE_ERR_INVALID_ARG, "params are not finite or s <= 0");
  *need = (size_t)h->h_ctl[2];
  return COLLAGE_OK;
}

static size_t with_slack(size_t need) { return std::max<size_t>(need + need / 2 + 256, 1024); }

static collage_status setup_level(collage_t h, int level) {
  drop_iter_graph(h);
  collage_status st = apply_level(h, level);
  if (st) return st;
  Dev& d = h->d;
  CK(h, prepare_dilate(h->opt.n_dilations));
  cudaStream_t s = h->cap_stream;
  CK(h, cudaMemsetAsync(h->ctl, 0, sizeof(int), s));  // clear latched status
  CK(h, enqueue_level_switch(d, s));
  // size the pair buffers from the current params
  size_t need = 0;
  st = probe_pairs(h, s, &need);
  if (st) return st;
  st = ensure_pairs(h, with_slack(need));
  if (st) return st;
  set_grids(h);
  h->level = level;
  return COLLAGE_OK;
}

// --------------------------------------------------------------------------------------------
// One iteration: transform -> bin -> raster fwd (+ losses) -> dilation -> adjoint -> loss -> Adam
// --------------------------------------------------------------------------------------------
// A named NVTX range around each kernel launch of an iteration (the checked build only; the
// ranges show in profilers that record NVTX, e.g. ncu --nvtx).  With COLLAGE_TRACE=1 in the
// environment the checked build also names each launch on stderr before it is made (with
// CUDA_LAUNCH_BLOCKING=1 the last name printed is the kernel that did not return).
struct LaunchRange {
#ifdef COLLAGE_CHECKED
  explicit LaunchRange(const char* name) {
    static const bool trace = getenv("COLLAGE_TRACE") && getenv("COLLAGE_TRACE")[0] == '1';
    if (trace) fprintf(stderr, "collage launch %s\n", name);
    nvtxRangePushA(name);
  }
  ~LaunchRange() { nvtxRangePop(); }
#else
  explicit LaunchRange(const char*) {}
#endif
};

static cudaError_t enqueue_iter(collage_t h, cudaStream_t s, int mode, float* out_bw, float* out_tau,
                                cudaEvent_t* ev = nullptr) {
  const Dev& d = h->d;
  const bool bwd = mode != kRender;
  const bool dil = bwd && d.L.gamma != 0.0f && d.L.n_dil > 0;
  cudaError_t e;
#define STEP_(x)                      \
  if ((e = (x)) != cudaSuccess) return e;
#define LAUNCH_(name, x) \
  {                      \
    LaunchRange r_(name); \
    STEP_(x);            \
  }
#define MARK_(i) \
  if (ev) STEP_(cudaEventRecord(ev[i], s));
  MARK_(0);
  LAUNCH_("k_transform", launch_transform(d, s, bwd && !d.deterministic));
  MARK_(1);
  MARK_(2);
  LAUNCH_("k_raster_chunks", launch_raster_fwd(d, s, h->pair_grid, h->tile_grid, out_bw, out_tau, 1));
  MARK_(3);
  LAUNCH_("k_composite", launch_raster_fwd(d, s, h->pair_grid, h->tile_grid, out_bw, out_tau, 2));
  MARK_(4);
  // the loss assembly needs only the composite's and the distribution term's partials: it runs on
  // a side stream beside the distribution adjoint and the raster adjoint (joined at the end of
  // the iteration); under stage timing it stays on the main stream
  const bool side = bwd && !ev;
  if (dil) LAUNCH_("k_dilate_fwd", launch_dilate(d, s, false));
  if (side) {
    STEP_(cudaEventRecord(h->ev_fork, s));
    STEP_(cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0));
    LAUNCH_("k_loss", launch_loss(d, h->aux_stream));
    STEP_(cudaEventRecord(h->ev_join, h->aux_stream));
  }
  if (dil) LAUNCH_("k_dilate_bwd", launch_dilate(d, s, true));
  MARK_(5);
  // in step mode the last block of the last gradient kernel marks this iteration's Adam step
  // pending; the next transform (or a flush before params are read) applies it
  const bool mark = mode == kStep;
  if (bwd) LAUNCH_("k_raster_bwd", launch_raster_bwd(d, s, h->bwd_grid, mark && !d.deterministic));
  MARK_(6);
  if (bwd && d.deterministic) LAUNCH_("k_grad_reduce", launch_grad_reduce(d, s, mark));
  MARK_(7);
  if (bwd && !side) LAUNCH_("k_loss", launch_loss(d, s));
  MARK_(8);
  // outline fitting: the points' gradient, and in step mode their Adam step and new outlines
  if (bwd && d.fit) LAUNCH_("k_ctrl_step", launch_ctrl_step(d, s, mode == kStep ? 1 : 0));
  if (side) STEP_(cudaStreamWaitEvent(s, h->ev_join, 0));
  MARK_(9);
#undef STEP_
#undef LAUNCH_
#undef MARK_
  return cudaSuccess;
}

static collage_status ensure_graph(collage_t h) {
  if (h->graph) return COLLAGE_OK;
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_iter(h, h->cap_stream, kStep, nullptr, nullptr);
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, e, "capture");
  }
  CK(h, e2);
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  CK(h, e);
  return COLLAGE_OK;
}

// The host-buffer step's graph: one iteration whose transform takes the params from the mapped
// input buffer h_in (so no copy precedes it), then the kernel that applies the Adam step and gathers
// params, loss terms and control words into the mapped h_stage.  Needs both mapped buffers.
static collage_status ensure_host_graph(collage_t h) {
  if (h->host_graph) return COLLAGE_OK;
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  h->d.q_in = h->h_in_dev;
  cudaError_t e = enqueue_iter(h, h->cap_stream, kStep, nullptr, nullptr);
  h->d.q_in = nullptr;
  if (e == cudaSuccess) e = launch_adam_flush(h->d, h->cap_stream, h->h_stage_dev);
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, e, "capture");
  }
  CK(h, e2);
  e = cudaGraphInstantiate(&h->host_graph, g, 0);
  cudaGraphDestroy(g);
  CK(h, e);
  return COLLAGE_OK;
}

// After a batch of work: check the latched status; grow the pair buffers when the last binning
// used more than 3/4 of them.  Returns OVERFLOW if the batch overflowed (caller re-runs).
static collage_status check_and_grow(collage_t h, cudaStream_t s, bool* overflowed) {
  *overflowed = false;
  collage_status st = read_ctl(h, s);
  if (st) return st;
  const int status = h->h_ctl[0];
  const size_t need = (size_t)h->h_ctl[2];
  if (status & kStatusInternal) return fail(h, COLLAGE_ERR_STATE, "internal bounds check failed");
  if (status & kStatusBadParam) {
    CK(h, cudaMemsetAsync(h->ctl, 0, sizeof(int), s));
    return fail(h, COLLAGE_ERR_INVALID_ARG, "params became non-finite or s <= 0");
  }
  if (status & (kStatusOverflow | kStatusTileCap)) {
    // void bins: the tiles' lists are cleared, then the pair buffers or the lists regrown
    *overflowed = true;
    int fullest = 0;
    if (status & kStatusTileCap) {
      // the emission counts on past the capacity: the fullest list's length, read before the
      // counts are cleared, sizes the lists in one regrow
      std::vector<int> cnt((size_t)h->d.total_tiles);
      CK(h, cudaMemcpyAsync(cnt.data(), h->d.tile_n, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, s));
      CK(h, cudaStreamSynchronize(s));
      for (int c : cnt) fullest = std::max(fullest, c);
    }
    CK(h, cudaMemsetAsync(h->ctl, 0, sizeof(int), s));
    CK(h, cudaMemsetAsync(h->d.tile_n, 0, sizeof(int) * h->tile_cap, s));
    CK(h, cudaStreamSynchronize(s));
    if (status & kStatusTileCap) {
      if (fullest >= (1 << 20)) return fail(h, COLLAGE_ERR_OVERFLOW, "a tile lists more than 2^20 pairs");
      int per_tile = 2 * h->d.tile_cap;  // at least doubled; past 3/4 full at the fullest list
      while (per_tile * 3 < fullest * 4) per_tile *= 2;
      collage_status st2 = ensure_tile_lists(h, per_tile);
      if (st2) return st2;
    }
    if (status & kStatusOverflow) {
      if (need + need / 2 + 256 > 0x7fffffff / 2) return fail(h, COLLAGE_ERR_OVERFLOW, "bin pairs exceed 2^30");
      return ensure_pairs(h, need + need / 2 + 256);
    }
    return COLLAGE_OK;
  }
  if (h->h_ctl[17] * 4 > h->d.tile_cap * 3) {  // the fullest tile list used more than 3/4
    collage_status st2 = ensure_tile_lists(h, 2 * h->d.tile_cap);
    if (st2) return st2;
  }
  if (need * 4 > h->pair_cap * 3) return ensure_pairs(h, need + need / 2 + 256);
  return COLLAGE_OK;
}

static collage_status run_checked(collage_t h, cudaStream_t s, int mode, float* out_bw, float* out_tau) {
  for (int attempt = 0; attempt < 4; ++attempt) {
    CK(h, enqueue_iter(h, s, mode, out_bw, out_tau));
    bool over = false;
    collage_status st = check_and_grow(h, s, &over);
    if (st) return st;
    if (!over) return COLLAGE_OK;
  }
  return fail(h, COLLAGE_ERR_OVERFLOW, "bin capacity kept overflowing");
}

// --------------------------------------------------------------------------------------------
// C ABI
// --------------------------------------------------------------------------------------------
extern "C" collage_status collage_create(const collage_problem* probs, int n_probs,
                                         const collage_options* opt, collage_t* out) {
  if (!out) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!probs || n_probs < 1) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "need n_probs >= 1 problems");
  collage_options o;
  if (opt) o = *opt;
  else collage_default_options(&o);
  std::string m = check_options(o);
  if (!m.empty()) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "options: " + m);
  long long total_e = 0;
  for (int p = 0; p < n_probs; ++p) {
    m = check_problem(probs[p], p, o);
    if (!m.empty()) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, m);
    total_e += probs[p].n_elems;
  }
  if (total_e > (1LL << 26)) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "too many elements");

  collage_t h = new collage_s();
  h->opt = o;
  if (h->opt.tile == 0) h->opt.tile = 16;  // the autotuner may change it later
  h->P = n_probs;
  h->prob_elem_base.push_back(0);
  h->prob_ring_base.push_back(0);
  h->ring_off.push_back(0);
  std::vector<float4> q;
  std::vector<uchar4> tr;
  for (int p = 0; p < n_probs; ++p) {
    const collage_problem& pr = probs[p];
    if (pr.trainable) h->has_trainable = true;
  }
  for (int p = 0; p < n_probs; ++p) {
    const collage_problem& pr = probs[p];
    for (int e = 0; e < pr.n_elems; ++e) {
      h->elem_prob.push_back(p);
      h->elem_voff.push_back((int)h->vloc.size());
      h->elem_coff.push_back((int)h->ctrl.size());
      h->elem_cubic.push_back(pr.kind[e] == COLLAGE_CUBIC_PATH ? 1 : 0);
      for (int k = pr.pt_off[e]; k < pr.pt_off[e + 1]; ++k)
        h->ctrl.push_back(make_float2(pr.pts[2 * k], pr.pts[2 * k + 1]));
      h->elem_closed.push_back(pr.kind[e] == COLLAGE_POLYLINE ? 0 : 1);
      h->elem_hw.push_back(pr.kind[e] == COLLAGE_POLYLINE && pr.stroke_hw ? pr.stroke_hw[e] : 0.0f);
      float rb = 0.0f;
      flatten(pr, e, o.segs_per_cubic, h->vloc, rb);
      h->elem_rbin.push_back(rb);
      const float* pp = pr.params0 + 4 * e;
      q.push_back(make_float4(pp[0], pp[1], pp[2], pp[3]));
      if (h->has_trainable) {
        const unsigned char* t = pr.trainable ? pr.trainable + 4 * e : nullptr;
        tr.push_back(t ? make_uchar4(t[0] != 0, t[1] != 0, t[2] != 0, t[3] != 0) : make_uchar4(1, 1, 1, 1));
      }
    }
    h->prob_elem_base.push_back((int)h->elem_prob.size());
    for (int r = 0; r < pr.n_rings; ++r) {
      for (int k = pr.ring_off[r]; k < pr.ring_off[r + 1]; ++k) {
        h->ring_pts.push_back(pr.ring_pts[2 * k]);
        h->ring_pts.push_back(pr.ring_pts[2 * k + 1]);
      }
      h->ring_off.push_back((int)(h->ring_pts.size() / 2));
    }
    h->prob_ring_base.push_back((int)h->ring_off.size() - 1);
    h->prob_grid.push_back(pr.grid ? pr.grid : o.level_res[o.n_levels - 1]);
  }
  h->elem_voff.push_back((int)h->vloc.size());
  h->elem_coff.push_back((int)h->ctrl.size());
  h->N = (int)h->elem_prob.size();
  h->V = (int)h->vloc.size();

  collage_status st = COLLAGE_OK;
  auto bail = [&](collage_status s2) {
    g_create_error = h->err;
    delete h;
    return s2;
  };
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) {
    cuda_fail(h, ce, "cudaGetDevice");
    return bail(COLLAGE_ERR_CUDA);
  }
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  if (h->sms < 1) h->sms = 1;
  Dev& d = h->d;
  d.n_elems = h->N;
  d.n_probs = h->P;
  d.max_segs = 0;
  for (int e = 0; e < h->N; ++e) d.max_segs = std::max(d.max_segs, h->elem_voff[e + 1] - h->elem_voff[e]);
  d.tile = h->opt.tile;
  d.emit_threads = 128;
  d.chunk_tiles = kChunkPx / d.tile;
  d.deterministic = o.deterministic ? 1 : 0;
  d.pdl = o.overlap_launches ? 1 : 0;
  d.lr = o.lr;
  d.b1 = o.beta1;
  d.b2 = o.beta2;
  d.eps = o.eps;
  d.s_min = o.s_min;
  d.s_max = o.s_max;
  d.L.alpha = o.alpha;
  d.L.beta = o.beta;
  d.L.gamma = o.gamma;
  d.L.delta = o.delta_down;
  d.L.force_kind = o.force_kind;
  d.L.fx = o.force_x;
  d.L.fy = o.force_y;
  d.L.tau = o.tau;
  d.L.w_in = o.w_in;
  d.L.w_out = o.w_out;
  d.L.n_dil = o.n_dilations;
  for (int k = 0; k < kMaxDil; ++k) d.L.dil_w[k] = o.dil_weight[k];
  d.L.pad_px = o.pad_px;
  d.L.rho_px = o.rho_px;
#define CKC(x)                                   \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) {                     \
      return bail(cuda_fail(h, e_, #x));         \
    }                                            \
  } while (0)
  int* p_elem_prob;
  int* p_elem_voff;
  uint8_t* p_closed;
  float* p_hw;
  float* p_rbin;
  float2* p_vloc;
  int* p_peb;
  double* p_ring;
  int* p_roff;
  int* p_prb;
  CKC(upload(h->owned, p_elem_prob, h->elem_prob));
  CKC(upload(h->owned, p_elem_voff, h->elem_voff));
  CKC(upload(h->owned, p_closed, h->elem_closed));
  CKC(upload(h->owned, p_hw, h->elem_hw));
  CKC(upload(h->owned, p_rbin, h->elem_rbin));
  CKC(upload(h->owned, p_vloc, h->vloc));
  CKC(upload(h->owned, p_peb, h->prob_elem_base));
  CKC(upload(h->owned, p_ring, h->ring_pts));
  CKC(upload(h->owned, p_roff, h->ring_off));
  CKC(upload(h->owned, p_prb, h->prob_ring_base));
  d.elem_prob = p_elem_prob;
  d.elem_voff = p_elem_voff;
  d.elem_closed = p_closed;
  d.elem_hw = p_hw;
  d.elem_rbin = p_rbin;
  d.vloc = p_vloc;
  d.prob_elem_base = p_peb;
  d.ring_pts = p_ring;
  d.ring_off = p_roff;
  d.prob_ring_base = p_prb;
  {
    // the points, and for fit_controls their Adam state, gradient and the per-vertex gradient
    int* p_coff;
    uint8_t* p_cubic;
    CKC(upload(h->owned, p_coff, h->elem_coff));
    CKC(upload(h->owned, p_cubic, h->elem_cubic));
    CKC(upload(h->owned, d.ctrl, h->ctrl));
    d.elem_coff = p_coff;
    d.elem_cubic = p_cubic;
    d.spc = o.segs_per_cubic;
    d.fit = o.fit_controls ? 1 : 0;
    const size_t nc = h->ctrl.size();
    CKC(dmalloc(h->owned, d.dctrl, nc));
    CKC(cudaMemset(d.dctrl, 0, sizeof(float2) * nc));
    if (d.fit) {
      CKC(dmalloc(h->owned, d.ctrl_m, nc));
      CKC(dmalloc(h->owned, d.ctrl_v, nc));
      CKC(dmalloc(h->owned, d.dv, h->V));
      CKC(cudaMemset(d.ctrl_m, 0, sizeof(float2) * nc));
      CKC(cudaMemset(d.ctrl_v, 0, sizeof(float2) * nc));
      CKC(cudaMemset(d.dv, 0, sizeof(float2) * h->V));
    }
  }
  CKC(upload(h->owned, d.q, q));
  CKC(dmalloc(h->owned, d.m, h->N));
  CKC(dmalloc(h->owned, d.v, h->N));
  CKC(cudaMemset(d.m, 0, sizeof(float4) * h->N));
  CKC(cudaMemset(d.v, 0, sizeof(float4) * h->N));
  if (h->has_trainable) {
    uchar4* p_tr;
    CKC(upload(h->owned, p_tr, tr));
    d.trainable = p_tr;
  }
  CKC(dmalloc(h->owned, d.segA, h->V));
  CKC(dmalloc(h->owned, d.segB, h->V));
  CKC(dmalloc(h->owned, d.segS, h->V));
  CKC(dmalloc(h->owned, d.tpx, h->N));
  CKC(dmalloc(h->owned, d.bbox, h->N));
  CKC(dmalloc(h->owned, d.rect, h->N));
  CKC(dmalloc(h->owned, d.dq, h->N));
  CKC(cudaMemset(d.dq, 0, sizeof(float4) * h->N));
  CKC(dmalloc(h->owned, d.loss_terms, 5 * h->P));
  CKC(cudaMemset(d.loss_terms, 0, sizeof(float) * 5 * h->P));
  CKC(dmalloc(h->owned, d.paths, 4));
  CKC(cudaMemset(d.paths, 0, sizeof(unsigned long long) * 4));
  CKC(dmalloc(h->owned, h->ctl, kCtlWords));
  CKC(cudaMemset(h->ctl, 0, sizeof(int) * kCtlWords));
  CKC(dmalloc(h->owned, d.elem_pbase, h->N));
  d.status = h->ctl;
  d.step = h->ctl + 1;
  d.total_pairs = h->ctl + 2;
  d.pending = h->ctl + 3;
  d.work = h->ctl + 4;
  d.sched_base = h->ctl + 12;
  d.chunk_count = h->ctl + 13;  // [13], [14]
  d.pair_need = h->ctl + 15;
  d.tile_max = h->ctl + 17;
  d.tile_cap = 16;  // pairs per tile list (doubled when a tile outgrows it)
  CKC(cudaMallocHost(&h->h_ctl, kCtlWords * sizeof(int)));
  std::memset(h->h_ctl, 0, kCtlWords * sizeof(int));
  CKC(dmalloc(h->owned, h->d_stage, stage_floats(h)));
  CKC(cudaHostAlloc(&h->h_stage, sizeof(float) * stage_floats(h), cudaHostAllocMapped));
  if (cudaHostGetDevicePointer(&h->h_stage_dev, h->h_stage, 0) != cudaSuccess) {
    h->h_stage_dev = nullptr;
    cudaGetLastError();
  }
  CKC(cudaHostAlloc(&h->h_in, sizeof(float4) * std::max<size_t>(h->N, 1), cudaHostAllocMapped));
  if (cudaHostGetDevicePointer(&h->h_in_dev, h->h_in, 0) != cudaSuccess) {
    h->h_in_dev = nullptr;
    cudaGetLastError();
  }
  CKC(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CKC(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
  CKC(cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking));
  CKC(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CKC(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
#undef CKC
  st = build_levels(h);
  if (st) return bail(st);
  st = setup_level(h, 0);
  if (st) return bail(st);
  *out = h;
  return COLLAGE_OK;
}

extern "C" void collage_destroy(collage_t h) {
  if (!h) return;
  cudaDeviceSynchronize();
  delete h;
}

extern "C" const char* collage_last_error(collage_t h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" collage_status collage_set_level(collage_t h, int level) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  if (level < 0 || level >= h->opt.n_levels) return fail(h, COLLAGE_ERR_INVALID_ARG, "level out of range");
  CK(h, cudaDeviceSynchronize());
  return setup_level(h, level);
}

extern "C" collage_status collage_render(collage_t h, void* stream, float* d_img_bw, float* d_img_tau) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  return run_checked(h, (cudaStream_t)stream, kRender, d_img_bw, d_img_tau);
}

extern "C" collage_status collage_loss_backward(collage_t h, void* stream, float* d_loss_terms,
                                                float* d_dparams) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  collage_status st = run_checked(h, s, kLossBwd, nullptr, nullptr);
  if (st) return st;
  if (d_loss_terms)
    CK(h, cudaMemcpyAsync(d_loss_terms, h->d.loss_terms, sizeof(float) * 5 * h->P, cudaMemcpyDeviceToDevice, s));
  if (d_dparams) CK(h, launch_copy_grad(h->d, s, d_dparams));
  return COLLAGE_OK;
}

// Enqueues n iterations in step mode: graph replays or eager launches.
static collage_status enqueue_steps(collage_t h, cudaStream_t s, int n) {
  if (h->opt.use_graphs) {
    collage_status st = ensure_graph(h);
    if (st) return st;
    for (int i = 0; i < n; ++i) CK(h, cudaGraphLaunch(h->graph, s));
  } else {
    for (int i = 0; i < n; ++i) CK(h, enqueue_iter(h, s, kStep, nullptr, nullptr));
  }
  return COLLAGE_OK;
}

extern "C" collage_status collage_step(collage_t h, void* stream, int n_iters) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  if (n_iters < 0) return fail(h, COLLAGE_ERR_INVALID_ARG, "n_iters must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  int remaining = n_iters;
  collage_status st = remaining > 0 && !h->ctl_current ? read_ctl(h, s) : COLLAGE_OK;
  if (st) return st;
  for (int attempt = 0; remaining > 0 && attempt < 8; ++attempt) {
    const int step0 = h->h_ctl[1];
    st = enqueue_steps(h, s, remaining);
    if (st) return st;
    bool over = false;
    st = check_and_grow(h, s, &over);  // reads the status and the step counter
    if (st) return st;
    remaining -= h->h_ctl[1] - step0;
    if (!over && remaining > 0) return fail(h, COLLAGE_ERR_STATE, "iterations went missing");
  }
  if (remaining > 0) return fail(h, COLLAGE_ERR_OVERFLOW, "bin capacity kept overflowing");
  return COLLAGE_OK;
}

extern "C" collage_status collage_step_async(collage_t h, void* stream, int n_iters) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  if (n_iters < 0) return fail(h, COLLAGE_ERR_INVALID_ARG, "n_iters must be >= 0");
  if (n_iters > 0) h->ctl_current = false;
  return enqueue_steps(h, (cudaStream_t)stream, n_iters);
}

// --------------------------------------------------------------------------------------------
// The level schedule (Sec. 4.3) as one CUDA graph: per level the level switch, then a WHILE node
// whose body is U iterations, U the largest divisor of the level's count up to kSchedUnroll (so
// the loop ends on the level's target); the loop conditions are set on the device (csrc/sched.cu).
constexpr int kSchedUnroll = 10;

// --------------------------------------------------------------------------------------------
static cudaError_t capture_schedule(collage_t h, int start, cudaStream_t s) {
  const collage_options& o = h->opt;
  cudaError_t e = launch_sched_begin(h->d, s);
  int target = 0;
  for (int l = start; l < o.n_levels && e == cudaSuccess; ++l) {
    if (apply_level(h, l) != COLLAGE_OK) return cudaErrorInvalidValue;  // tables exist: host only
    set_grids(h);
    const Dev& d = h->d;
    target += o.level_iters[l];
    e = enqueue_level_switch(d, s);
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphConditionalHandle cond = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, g, 0, 0);
    if (e == cudaSuccess) e = launch_sched_cond(d, s, cond, target);
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) break;
    // the loop body: U iterations, then the condition for the next pass (one body relaunch and
    // one condition kernel per U iterations; a status latched inside the body makes its later
    // kernels return without stepping, so the loop still stops on the iteration that failed)
    const int n_l = o.level_iters[l];
    int U = 1;
    for (int u = std::min(n_l, kSchedUnroll); u > 1; --u)
      if (n_l % u == 0) {
        U = u;
        break;
      }
    cudaStream_t b = h->body_stream;
    e = cudaStreamBeginCaptureToGraph(b, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    cudaError_t eb = cudaSuccess;
    for (int u = 0; u < U && eb == cudaSuccess; ++u) eb = enqueue_iter(h, b, kStep, nullptr, nullptr);
    if (eb == cudaSuccess) eb = launch_sched_cond(d, b, cond, target);
    cudaGraph_t body = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b, &body);
    e = eb != cudaSuccess ? eb : ee;
  }
  return e;
}

// Capacity for every level of a run from `start` (probed from the current params), then the
// capture.  Synchronises the device.
static collage_status build_schedule(collage_t h, int start) {
  const int cur = h->level;
  cudaStream_t s = h->cap_stream;
  CK(h, cudaDeviceSynchronize());
  size_t need = 0;
  collage_status st = COLLAGE_OK;
  for (int l = start; l < h->opt.n_levels && !st; ++l) {
    st = apply_level(h, l);
    size_t n = 0;
    if (!st) st = probe_pairs(h, s, &n);
    need = std::max(need, n);
  }
  collage_status st2 = apply_level(h, cur);
  if (st) return st;
  if (st2) return st2;
  if (with_slack(need) > h->pair_cap) {
    st = ensure_pairs(h, with_slack(need));
    if (st) return st;
  }
  if (h->sched) cudaGraphExecDestroy(h->sched);
  h->sched = nullptr;
  h->sched_start = -1;
  CK(h, prepare_dilate(h->opt.n_dilations));
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const cudaError_t e = capture_schedule(h, start, s);
  const cudaError_t e2 = cudaStreamEndCapture(s, &g);
  st = apply_level(h, cur);  // the current level's view again
  set_grids(h);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, e != cudaSuccess ? e : e2, "schedule capture");
  }
  if (st) {
    cudaGraphDestroy(g);
    return st;
  }
  const cudaError_t ei = cudaGraphInstantiate(&h->sched, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    h->sched = nullptr;
    return cuda_fail(h, ei, "schedule instantiate");
  }
  h->sched_start = start;
  return COLLAGE_OK;
}

// The host-driven schedule: level setup on the host, then the level's iterations.
static collage_status run_schedule_host(collage_t h, void* stream, int level, int done_in_level) {
  for (int l = level; l < h->opt.n_levels; ++l) {
    if (l != h->level) {
      collage_status st = collage_set_level(h, l);
      if (st) return st;
    }
    collage_status st = collage_step(h, stream, h->opt.level_iters[l] - (l == level ? done_in_level : 0));
    if (st) return st;
  }
  return COLLAGE_OK;
}

extern "C" collage_status collage_run_schedule(collage_t h, void* stream) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  const collage_options& o = h->opt;
  const int L = o.n_levels, start = std::max(h->level, 0);
  if (!o.use_graphs) return run_schedule_host(h, stream, start, 0);
  cudaStream_t s = (cudaStream_t)stream;
  bool over = false;
  collage_status st = check_and_grow(h, s, &over);  // nothing latched; the step count read
  if (st) return st;
  if (!h->sched || h->sched_start != start) {
    st = build_schedule(h, start);
    if (st) return st;
    st = check_and_grow(h, s, &over);
    if (st) return st;
  }
  const int step0 = h->h_ctl[1];
  CK(h, cudaGraphLaunch(h->sched, s));
  h->ctl_current = false;
  st = read_ctl(h, s);
  if (st) return st;
  const int done = h->h_ctl[1] - step0;
  int total = 0;
  for (int l = start; l < L; ++l) total += o.level_iters[l];
  // the device now holds the last level that ran (or the last level): the host view follows
  drop_iter_graph(h);
  h->level = -1;
  if (done == total && !(h->h_ctl[0] & (kStatusVoid | kStatusInternal))) {
    st = apply_level(h, L - 1);
    if (st) return st;
    set_grids(h);
    h->level = L - 1;
    return check_and_grow(h, s, &over);  // grows the pair buffers if the last level used > 3/4
  }
  // stopped early (a bin overflow, or params became non-finite): resume on the host path from the
  // iteration that did not complete
  st = check_and_grow(h, s, &over);
  if (st) return st;
  int l = start, acc = 0;
  while (l < L - 1 && acc + o.level_iters[l] <= done) acc += o.level_iters[l++];
  return run_schedule_host(h, stream, l, done - acc);
}

extern "C" collage_status collage_step_host(collage_t h, void* stream, int n_iters,
                                            const float* h_params_in, float* h_params_out,
                                            float* h_loss_out) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  if (n_iters < 0) return fail(h, COLLAGE_ERR_INVALID_ARG, "n_iters must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  collage_status st = h->ctl_current ? COLLAGE_OK : read_ctl(h, s);
  if (st) return st;
  const int step0 = h->h_ctl[1];
  // one iteration with params in: one graph launch (its transform reads them from the mapped
  // input buffer and takes a pending step's moments; its last kernel writes the mapped output)
  const bool host_graph = h_params_in && n_iters == 1 && h->opt.use_graphs && h->h_in_dev && h->h_stage_dev;
  if (host_graph) {
    st = ensure_host_graph(h);
    if (st) return st;
    std::memcpy(h->h_in, h_params_in, sizeof(float4) * h->N);
    CK(h, cudaGraphLaunch(h->host_graph, s));
  } else {
    if (h_params_in) {
      // a pending step belongs to the old params (none is pending right after this call's flush)
      if (h->h_ctl[3] != 0) CK(h, launch_adam_flush(h->d, s));
      CK(h, cudaMemcpyAsync(h->d.q, h_params_in, sizeof(float4) * h->N, cudaMemcpyHostToDevice, s));
    }
    // one host round trip when nothing overflows: the steps, then one kernel that applies the
    // last Adam step and gathers the params, the loss terms and the control words, one copy of
    // those to pinned memory, and one synchronisation
    st = enqueue_steps(h, s, n_iters);
    if (st) return st;
  }
  auto copy_out = [&](bool launched) -> collage_status {
    if (launched) {
    } else if (h->h_stage_dev) {
      CK(h, launch_adam_flush(h->d, s, h->h_stage_dev));
    } else {
      CK(h, launch_adam_flush(h->d, s, h->d_stage));
      CK(h, cudaMemcpyAsync(h->h_stage, h->d_stage, sizeof(float) * stage_floats(h), cudaMemcpyDeviceToHost, s));
    }
    CK(h, cudaStreamSynchronize(s));
    const float* tail = h->h_stage + 4 * (size_t)h->N;
    if (h_params_out) std::memcpy(h_params_out, h->h_stage, sizeof(float4) * h->N);
    if (h_loss_out) std::memcpy(h_loss_out, tail, sizeof(float) * 5 * h->P);
    std::memcpy(h->h_ctl, tail + 5 * h->P, kCtlWords * sizeof(int));
    h->ctl_current = true;
    return COLLAGE_OK;
  };
  st = copy_out(host_graph);
  if (st) return st;
  const int status = h->h_ctl[0], done = h->h_ctl[1] - step0;
  if (!(status & (kStatusVoid | kStatusInternal)) && done == n_iters &&
      (size_t)h->h_ctl[2] * 4 <= h->pair_cap * 3 && h->h_ctl[17] * 4 <= h->d.tile_cap * 3)
    return COLLAGE_OK;
  // an overflow (or a status to report): the synchronous path regrows and runs the rest
  bool over = false;
  st = check_and_grow(h, s, &over);
  if (st) return st;
  if (done < n_iters) {
    st = collage_step(h, stream, n_iters - done);
    if (st) return st;
    st = copy_out(false);
    if (st) return st;
  }
  return COLLAGE_OK;
}

extern "C" collage_status collage_get_loss(collage_t h, void* stream, float* d_loss_terms) {
  if (!h || !d_loss_terms) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  CK(h, cudaMemcpyAsync(d_loss_terms, h->d.loss_terms, sizeof(float) * 5 * h->P, cudaMemcpyDeviceToDevice,
                        (cudaStream_t)stream));
  return COLLAGE_OK;
}

extern "C" collage_status collage_get_params(collage_t h, void* stream, float* d_params) {
  if (!h || !d_params) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  CK(h, launch_adam_flush(h->d, (cudaStream_t)stream));
  CK(h, cudaMemcpyAsync(d_params, h->d.q, sizeof(float4) * h->N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return COLLAGE_OK;
}

extern "C" collage_status collage_set_params(collage_t h, void* stream, const float* d_params) {
  if (!h || !d_params) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  CK(h, launch_adam_flush(h->d, (cudaStream_t)stream));  // the step belongs to the old params
  CK(h, cudaMemcpyAsync(h->d.q, d_params, sizeof(float4) * h->N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return COLLAGE_OK;
}

extern "C" collage_status collage_get_controls(collage_t h, void* stream, float* d_pts) {
  if (!h || !d_pts) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  CK(h, cudaMemcpyAsync(d_pts, h->d.ctrl, sizeof(float2) * h->ctrl.size(), cudaMemcpyDeviceToDevice,
                        (cudaStream_t)stream));
  return COLLAGE_OK;
}

extern "C" collage_status collage_set_controls(collage_t h, void* stream, const float* d_pts) {
  if (!h || !d_pts) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(h, cudaMemcpyAsync(h->d.ctrl, d_pts, sizeof(float2) * h->ctrl.size(), cudaMemcpyDeviceToDevice, s));
  CK(h, launch_ctrl_step(h->d, s, 2));  // new outlines and bin radii
  return COLLAGE_OK;
}

extern "C" collage_status collage_get_control_grad(collage_t h, void* stream, float* d_dpts) {
  if (!h || !d_dpts) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  CK(h, cudaMemcpyAsync(d_dpts, h->d.dctrl, sizeof(float2) * h->ctrl.size(), cudaMemcpyDeviceToDevice,
                        (cudaStream_t)stream));
  return COLLAGE_OK;
}

extern "C" collage_status collage_get_state(collage_t h, void* stream, float* d_state, int* h_step,
                                            int* h_level) {
  if (!h || !d_state) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = sizeof(float4) * h->N;
  CK(h, launch_adam_flush(h->d, s));
  CK(h, cudaMemcpyAsync(d_state, h->d.q, n, cudaMemcpyDeviceToDevice, s));
  CK(h, cudaMemcpyAsync((char*)d_state + n, h->d.m, n, cudaMemcpyDeviceToDevice, s));
  CK(h, cudaMemcpyAsync((char*)d_state + 2 * n, h->d.v, n, cudaMemcpyDeviceToDevice, s));
  collage_status st = read_ctl(h, s);
  if (st) return st;
  if (h_step) *h_step = h->h_ctl[1];
  if (h_level) *h_level = h->level;
  return COLLAGE_OK;
}

extern "C" collage_status collage_set_state(collage_t h, void* stream, const float* d_state, int h_step,
                                            int h_level) {
  if (!h || !d_state) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  if (h_step < 0) return fail(h, COLLAGE_ERR_INVALID_ARG, "step must be >= 0");
  if (h_level != h->level) {
    collage_status st = collage_set_level(h, h_level);
    if (st) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = sizeof(float4) * h->N;
  CK(h, cudaMemcpyAsync(h->d.q, d_state, n, cudaMemcpyDeviceToDevice, s));
  CK(h, cudaMemcpyAsync(h->d.m, (const char*)d_state + n, n, cudaMemcpyDeviceToDevice, s));
  CK(h, cudaMemcpyAsync(h->d.v, (const char*)d_state + 2 * n, n, cudaMemcpyDeviceToDevice, s));
  h->h_ctl[1] = h_step;
  CK(h, cudaMemcpyAsync(h->d.step, &h->h_ctl[1], sizeof(int), cudaMemcpyHostToDevice, s));
  CK(h, cudaMemsetAsync(h->d.pending, 0, sizeof(int), s));  // the state replaces everything
  CK(h, cudaStreamSynchronize(s));
  h->h_ctl[3] = 0;
  h->ctl_current = true;
  return COLLAGE_OK;
}

extern "C" collage_status collage_get_bins(collage_t h, void* stream, int* d_tile, int* d_elem, int cap,
                                           int* h_n) {
  if (!h || !h_n) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  collage_status st = read_ctl(h, s);
  if (st) return st;
  const int n = h->h_ctl[2];
  *h_n = n;
  if (!d_tile && !d_elem) return COLLAGE_OK;
  if (cap < n) return fail(h, COLLAGE_ERR_INVALID_ARG, "cap is smaller than the pair count");
  const size_t nt = (size_t)h->d.total_tiles, C = (size_t)h->d.tile_cap;
  std::vector<int> tm(nt), ts(nt * C), te, ee;
  CK(h, cudaMemcpy(tm.data(), h->d.tile_m, sizeof(int) * nt, cudaMemcpyDeviceToHost));
  CK(h, cudaMemcpy(ts.data(), h->d.tile_sorted, sizeof(int) * nt * C, cudaMemcpyDeviceToHost));
  te.reserve(n);
  ee.reserve(n);
  for (size_t t = 0; t < nt; ++t)
    for (int k = 0; k < tm[t] && k < (int)C; ++k) {
      te.push_back((int)t);
      ee.push_back(ts[t * C + k]);
    }
  if ((int)te.size() != n) return fail(h, COLLAGE_ERR_STATE, "tile lists disagree with the pair count");
  if (d_tile && n) CK(h, cudaMemcpy(d_tile, te.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  if (d_elem && n) CK(h, cudaMemcpy(d_elem, ee.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  return COLLAGE_OK;
}

extern "C" collage_status collage_stage_times(collage_t h, void* stream, int n_iters, float* h_ms) {
  if (!h || !h_ms || n_iters < 1) return fail(h, COLLAGE_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  constexpr int NE = COLLAGE_N_STAGES + 1;
  cudaEvent_t ev[NE];
  for (int i = 0; i < NE; ++i) CK(h, cudaEventCreate(&ev[i]));
  double acc[NE - 1] = {0};
  collage_status st = COLLAGE_OK;
  for (int it = 0; it < n_iters && !st; ++it) {
    cudaError_t e = enqueue_iter(h, s, kStep, nullptr, nullptr, ev);
    if (e != cudaSuccess) {
      st = cuda_fail(h, e, "enqueue");
      break;
    }
    e = cudaEventSynchronize(ev[NE - 1]);
    if (e != cudaSuccess) {
      st = cuda_fail(h, e, "sync");
      break;
    }
    for (int i = 0; i < NE - 1; ++i) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      acc[i] += ms;
    }
  }
  for (int i = 0; i < NE; ++i) cudaEventDestroy(ev[i]);
  if (st) return st;
  // events bracket the stages in COLLAGE_STAGE_* order
  for (int i = 0; i < COLLAGE_N_STAGES; ++i) h_ms[i] = (float)(acc[i] / n_iters);
  bool over = false;
  return check_and_grow(h, s, &over);
}

// --------------------------------------------------------------------------------------------
// Autotuner: raster tile, emission block size and the persistent grids of the emission, adjoint
// and composite kernels, timed on a captured graph of one loss + gradient iteration; the choice
// is cached per (level pixels, elements, pair density) for the process.
// --------------------------------------------------------------------------------------------
namespace {
struct TuneChoice {
  int tile, emit_threads, chunk_px;
  float fwd, bwd, comp;
};
std::mutex g_tune_mu;
std::map<std::tuple<long long, int, int, int>, TuneChoice> g_tune_cache;

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// A buffer of twice the L2 size, written before each timed replay so that every candidate starts
// from a cold cache, as a step does after the host or other work has used the device.
struct L2Evict {
  void* p = nullptr;
  size_t n = 0;
  ~L2Evict() {
    if (p) cudaFree(p);
  }
};
}  // namespace

// Applies a choice (tile change: new level tables and pair buffers).
static collage_status apply_choice(collage_t h, const TuneChoice& c) {
  const bool retile = c.tile != h->d.tile;
  h->d.tile = c.tile;
  h->opt.tile = c.tile;
  h->d.emit_threads = c.emit_threads;
  h->d.chunk_tiles = std::max(1, c.chunk_px / c.tile);
  h->fwd_mult = c.fwd;
  h->bwd_mult = c.bwd;
  h->comp_mult = c.comp;
  drop_graph(h);
  if (retile) return setup_level(h, h->level);
  set_grids(h);
  return COLLAGE_OK;
}

// Milliseconds per loss + gradient iteration (no Adam step) in the current configuration: a
// captured one-iteration graph, 3 replays to warm up, then three batches of `reps` replays, each
// timed alone after the L2 eviction write; the fastest batch's mean (the least disturbed by
// anything else on the device).  Timed warm and back to back, the replays favoured launch
// parameters whose gain reversed from a cold cache.
static collage_status time_config(collage_t h, cudaStream_t s, int reps, const L2Evict& ev2,
                                  float* ms) {
  collage_status st = run_checked(h, s, kLossBwd, nullptr, nullptr);  // regrows if needed
  if (st) return st;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  const cudaError_t e = enqueue_iter(h, h->cap_stream, kLossBwd, nullptr, nullptr);
  const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, e != cudaSuccess ? e : e2, "autotune capture");
  }
  const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  CK(h, ei);
  EventPair ev;
  cudaError_t er = cudaEventCreate(&ev.a);
  if (er == cudaSuccess) er = cudaEventCreate(&ev.b);
  for (int i = 0; i < 3 && er == cudaSuccess; ++i) {
    er = cudaMemsetAsync(ev2.p, 0, ev2.n, s);
    if (er == cudaSuccess) er = cudaGraphLaunch(ge, s);
  }
  float t = 1e30f;
  for (int batch = 0; batch < 3 && er == cudaSuccess; ++batch) {
    float tb = 0.0f;
    for (int i = 0; i < reps && er == cudaSuccess; ++i) {
      er = cudaMemsetAsync(ev2.p, 0, ev2.n, s);
      if (er == cudaSuccess) er = cudaEventRecord(ev.a, s);
      if (er == cudaSuccess) er = cudaGraphLaunch(ge, s);
      if (er == cudaSuccess) er = cudaEventRecord(ev.b, s);
      if (er == cudaSuccess) er = cudaEventSynchronize(ev.b);
      float ti = 0.0f;
      if (er == cudaSuccess) er = cudaEventElapsedTime(&ti, ev.a, ev.b);
      tb += ti;
    }
    t = std::min(t, tb);
  }
  cudaGraphExecDestroy(ge);
  CK(h, er);
  bool over = false;
  st = check_and_grow(h, s, &over);
  if (st) return st;
  if (over) return time_config(h, s, reps, ev2, ms);  // grown: time again
  *ms = t / reps;
  return COLLAGE_OK;
}

extern "C" collage_status collage_autotune(collage_t h, void* stream, float* h_best_ms) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const TuneChoice before{h->d.tile, h->d.emit_threads, h->d.chunk_tiles * h->d.tile, h->fwd_mult,
                          h->bwd_mult, h->comp_mult};
  // the key: pixels of the level, elements, and the pair density at 8-px tiles (half-octaves)
  long long pix = 0;
  for (int p = 0; p < h->P; ++p) pix += (long long)h->res[p] * h->res[p];
  const double tiles8 = std::max(1.0, (double)pix / 64.0);
  const double pairs = (double)std::max(h->h_ctl[2], 1) * (h->d.tile == 8 ? 1.0 : 4.0);
  const int density = (int)std::floor(2.0 * std::log2(1.0 + pairs / tiles8));
  const auto key = std::make_tuple(pix, h->N, density, h->opt.deterministic);
  L2Evict ev2;
  {
    int dev = 0, l2 = 0;
    CK(h, cudaGetDevice(&dev));
    CK(h, cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    ev2.n = std::max<size_t>(2 * (size_t)l2, (size_t)64 << 20);
    CK(h, cudaMalloc(&ev2.p, ev2.n));
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      collage_status st = apply_choice(h, it->second);
      if (st) return st;
      float ms = 0.0f;
      st = time_config(h, s, 10, ev2, &ms);
      if (st) return st;
      h->tuning.tile = it->second.tile;
      h->tuning.emit_threads = it->second.emit_threads;
      h->tuning.chunk_px = it->second.chunk_px;
      h->tuning.fwd_grid = it->second.fwd;
      h->tuning.bwd_grid = it->second.bwd;
      h->tuning.comp_grid = it->second.comp;
      h->tuning.best_ms = ms;
      h->tuning.trials = 0;
      h->tuning.from_cache = 1;
      if (h_best_ms) *h_best_ms = ms;
      return COLLAGE_OK;
    }
  }
  const int reps = 20;
  int trials = 0;
  TuneChoice best{16, 128, kChunkPx, 1.0f, 1.0f, 1.0f};
  float best_ms = 1e30f, default_ms = 0.0f;
  auto trial = [&](const TuneChoice& c, float* out) -> collage_status {
    collage_status st = apply_choice(h, c);
    if (!st) st = time_config(h, s, reps, ev2, out);
    ++trials;
    return st;
  };
  collage_status st = COLLAGE_OK;
  // the tile first (the defaults of everything else), then each launch parameter in turn
  for (int T : {16, 8}) {
    float ms = 0.0f;
    const TuneChoice c{T, 128, kChunkPx, 1.0f, 1.0f, 1.0f};
    if ((st = trial(c, &ms))) break;
    if (T == 16) default_ms = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  const float mults[3] = {0.5f, 1.0f, 2.0f};
  for (int dim = 0; dim < 5 && !st; ++dim) {
    const TuneChoice base = best;
    for (int k = 0; k < (dim <= 1 ? 2 : 3) && !st; ++k) {
      TuneChoice c = base;
      if (dim == 0) c.emit_threads = k == 0 ? 128 : 256;
      if (dim == 1) c.chunk_px = k == 0 ? kChunkPx : kChunkPx / 2;
      if (dim == 2) c.fwd = mults[k];
      if (dim == 3) c.bwd = mults[k];
      if (dim == 4) c.comp = mults[k];
      if (std::memcmp(&c, &base, sizeof(c)) == 0) continue;
      float ms = 0.0f;
      if ((st = trial(c, &ms))) break;
      if (ms < best_ms * 0.97f) {  // a change of launch parameter has to win clearly (3%:
        // smaller gains on the one-iteration graph do not carry to the whole step)
        best_ms = ms;
        best = c;
      }
    }
  }
  if (st) {  // leave the handle as it was
    apply_choice(h, before);
    return st;
  }
  st = apply_choice(h, best);
  if (st) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
  }
  h->tuning.tile = best.tile;
  h->tuning.emit_threads = best.emit_threads;
  h->tuning.chunk_px = best.chunk_px;
  h->tuning.fwd_grid = best.fwd;
  h->tuning.bwd_grid = best.bwd;
  h->tuning.comp_grid = best.comp;
  h->tuning.default_ms = default_ms;
  h->tuning.best_ms = best_ms;
  h->tuning.trials = trials;
  h->tuning.from_cache = 0;
  if (h_best_ms) *h_best_ms = best_ms;
  return COLLAGE_OK;
}

extern "C" collage_status collage_get_tuning(collage_t h, collage_tuning* out) {
  if (!h || !out) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  *out = h->tuning;
  out->tile = h->d.tile;
  out->emit_threads = h->d.emit_threads;
  out->chunk_px = h->d.chunk_tiles * h->d.tile;
  out->fwd_grid = h->fwd_mult;
  out->bwd_grid = h->bwd_mult;
  out->comp_grid = h->comp_mult;
  return COLLAGE_OK;
}

extern "C" collage_status collage_set_tuning(collage_t h, void* stream, const collage_tuning* c) {
  (void)stream;
  if (!h || !c) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  auto grid_ok = [](float m) { return m == 0.5f || m == 1.0f || m == 2.0f; };
  if ((c->tile != 8 && c->tile != 16) || (c->emit_threads != 128 && c->emit_threads != 256) ||
      (c->chunk_px != kChunkPx && c->chunk_px != kChunkPx / 2) || !grid_ok(c->fwd_grid) ||
      !grid_ok(c->bwd_grid) || !grid_ok(c->comp_grid))
    return fail(h, COLLAGE_ERR_INVALID_ARG, "tuning outside the searched values");
  CK(h, cudaDeviceSynchronize());
  const TuneChoice before{h->d.tile, h->d.emit_threads, h->d.chunk_tiles * h->d.tile, h->fwd_mult,
                          h->bwd_mult, h->comp_mult};
  const TuneChoice want{c->tile, c->emit_threads, c->chunk_px, c->fwd_grid, c->bwd_grid, c->comp_grid};
  collage_status st = apply_choice(h, want);
  if (st) {
    apply_choice(h, before);
    return st;
  }
  h->tuning = collage_tuning{};
  return COLLAGE_OK;
}

extern "C" collage_status collage_mat_init(collage_t h, void* stream, int* d_axis, float* d_width) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t np = (size_t)h->d.total_pix, al = 256;
  auto up = [&](size_t b) { return (b + al - 1) / al * al; };
  // gcol, D2, candidates, clearances (4 B per pixel each), placement order, candidate counts
  const size_t need = 4 * up(4 * np) + up(sizeof(int) * (size_t)h->N) + up(sizeof(int) * (size_t)h->P);
  if (need > h->mat_bytes) {
    CK(h, cudaDeviceSynchronize());
    if (h->mat_buf) cudaFree(h->mat_buf);
    h->mat_buf = nullptr;
    h->mat_bytes = 0;
    CK(h, cudaMalloc(&h->mat_buf, need));
    h->mat_bytes = need;
  }
  unsigned char* b = h->mat_buf;
  int* gcol = reinterpret_cast<int*>(b);
  unsigned* d2 = reinterpret_cast<unsigned*>(b + up(4 * np));
  int* cand = reinterpret_cast<int*>(b + 2 * up(4 * np));
  float* clear = reinterpret_cast<float*>(b + 3 * up(4 * np));
  int* order = reinterpret_cast<int*>(b + 4 * up(4 * np));
  int* n_cand = reinterpret_cast<int*>(b + 4 * up(4 * np) + up(sizeof(int) * (size_t)h->N));
  CK(h, launch_adam_flush(h->d, s));  // a pending step belongs to the old params
  int max_res = 1;
  for (int p = 0; p < h->P; ++p) max_res = std::max(max_res, h->res[p]);
  CK(h, launch_mat_init(h->d, s, max_res, gcol, d2, cand, n_cand, clear, order, d_axis, d_width));
  return COLLAGE_OK;
}

extern "C" collage_status collage_metrics(collage_t h, void* stream, double* h_metrics) {
  if (!h || !h_metrics) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t np = (size_t)h->d.total_pix;
  if (np > h->met_pix) {
    CK(h, cudaDeviceSynchronize());
    if (h->met_obj) cudaFree(h->met_obj);
    if (h->met_gcol) cudaFree(h->met_gcol);
    h->met_obj = nullptr;
    h->met_gcol = nullptr;
    h->met_pix = 0;
    CK(h, cudaMalloc(&h->met_obj, np));
    CK(h, cudaMalloc(&h->met_gcol, sizeof(int) * np));
    h->met_pix = np;
  }
  if (!h->met_cnt) CK(h, cudaMalloc(&h->met_cnt, sizeof(unsigned long long) * 5 * h->P));
  CK(h, launch_adam_flush(h->d, s));
  collage_status st = run_checked(h, s, kRender, nullptr, nullptr);
  if (st) return st;
  int max_res = 1;
  for (int p = 0; p < h->P; ++p) max_res = std::max(max_res, h->res[p]);
  CK(h, launch_metrics(h->d, s, h->met_obj, h->met_gcol, h->met_cnt, h->met_cnt + 4 * h->P, max_res));
  std::vector<unsigned long long> c(5 * (size_t)h->P);
  CK(h, cudaMemcpyAsync(c.data(), h->met_cnt, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  for (int p = 0; p < h->P; ++p) {
    const double in = (double)c[4 * p], shape = (double)c[4 * p + 1], over = (double)c[4 * p + 2],
                 out = (double)c[4 * p + 3], sum = (double)c[4 * h->P + p];
    const double free_px = shape - in, r = (double)h->res[p];
    double* m = h_metrics + 8 * p;
    m[0] = in;
    m[1] = shape;
    m[2] = over;
    m[3] = out;
    m[4] = shape > 0 ? in / shape : 0.0;
    m[5] = shape > 0 ? over / shape : 0.0;
    m[6] = shape > 0 ? out / shape : 0.0;
    m[7] = (in + out > 0 && free_px > 0) ? sum / free_px / (r * r) : 0.0;
  }
  return COLLAGE_OK;
}

extern "C" collage_status collage_get_info(collage_t h, collage_info* out) {
  if (!h || !out) return fail(h, COLLAGE_ERR_INVALID_ARG, "NULL argument");
  out->n_probs = h->P;
  out->n_elems = h->N;
  out->level = h->level;
  out->n_levels = h->opt.n_levels;
  out->tile = h->d.tile;
  out->total_pixels = h->d.total_pix;
  out->pair_capacity = h->d.cap;
  out->last_pairs = h->h_ctl ? h->h_ctl[2] : 0;
  // transform (with the previous Adam step and the pair slots), emission with signed distances,
  // composite, (2 dilation), raster bwd, (gradient reduce), loss
  const bool dil = h->d.L.gamma != 0.0f && h->d.L.n_dil > 0;
  out->kernels_per_iter = 3 + (dil ? 2 : 0) + 1 +
                         (h->d.deterministic ? 1 : 0) + 1 + (h->d.fit ? 1 : 0);
  unsigned long long paths[4] = {0, 0, 0, 0};
  CK(h, cudaDeviceSynchronize());
  CK(h, cudaMemcpy(paths, h->d.paths, sizeof(paths), cudaMemcpyDeviceToHost));
  out->path_row_fallback = (long long)paths[0];
  out->path_long_near = (long long)paths[1];
  out->path_wide_tile = (long long)paths[2];
  out->path_ring_chunk = (long long)paths[3];
  return COLLAGE_OK;
}

extern "C" collage_status collage_sync(collage_t h, void* stream) {
  if (!h) return fail(nullptr, COLLAGE_ERR_INVALID_ARG, "handle is NULL");
  bool over = false;
  collage_status st = check_and_grow(h, (cudaStream_t)stream, &over);
  if (st) return st;
  if (over) return fail(h, COLLAGE_ERR_OVERFLOW, "the last asynchronous call overflowed the bins; it was regrown, repeat the call");
  return COLLAGE_OK;
}
