/* libcollage -- GB300 (sm_103a) hot path of image-space collage and packing.
 *
 * Method: Wang & Lu, "Image-Space Collage and Packing with Differentiable Rendering"
 * (SIGGRAPH Conference Papers 2025, arXiv 2406.04008).  The collage problem (Sec. 3, Eq. 1) places
 * n vector items inside a container by optimising one similarity transform per item; items are
 * transformed (Eq. 2), rasterised with anti-aliased coverage, scored by image-space losses against
 * the rasterised container (Sec. 4.2, Eqs. 5-8, plus the downward or point force of Sec. 5) and updated by
 * gradient steps (Eq. 4, here Adam), coarse to fine over a resolution pyramid (Sec. 4.3).
 *
 * Conventions.  Unit-square world coordinates, y down.  Pixel (i, j) of an R x R grid has its
 * centre at ((j + 1/2)/R, (i + 1/2)/R).  Params are float32 (tx, ty, theta, s) per element, with
 * world point = R(theta) (s * local point) + (tx, ty).
 *
 * Pointers: names starting with d_ are device pointers (e.g. torch CUDA tensors), h_ are host
 * pointers, everything in collage_problem is host memory that is copied during collage_create.
 * Streams are cudaStream_t passed as void* (NULL = the legacy default stream).
 *
 * Errors: every call returns a collage_status; no call throws across the ABI.  Invalid arguments
 * are detected before any device work.  Errors found on the device during an asynchronous call
 * (bin-capacity overflow, a bounded wait that gave up) are latched in a device status word and
 * returned by the next synchronous call on the handle (collage_step, collage_sync).  The message of
 * the last failure of a handle is returned by collage_last_error.  A handle is not thread-safe.
 */
#ifndef COLLAGE_H
#define COLLAGE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef int collage_status;
#define COLLAGE_OK 0
#define COLLAGE_ERR_INVALID_ARG (-1) /* an argument failed validation; nothing was run */
#define COLLAGE_ERR_OOM (-2)         /* a device allocation failed */
#define COLLAGE_ERR_CUDA (-3)        /* a CUDA runtime call failed (message has the CUDA error) */
#define COLLAGE_ERR_OVERFLOW (-4)    /* a device capacity was exceeded and could not be regrown */
#define COLLAGE_ERR_TIMEOUT (-5)     /* a bounded device wait gave up */
#define COLLAGE_ERR_STATE (-6)       /* call not valid in the handle's current state */

typedef struct collage_s* collage_t;

/* Element kinds (Sec. 3 "Vector Representation"; polygons and polylines are the degenerate
 * cases the paper's examples also use: sketched paths and glyph strokes). */
#define COLLAGE_CUBIC_PATH 0 /* closed path of N cubic Beziers, 3N control points; curve k uses
                                points 3k, 3k+1, 3k+2 and 3k+3 (mod 3N) */
#define COLLAGE_POLYGON 1    /* closed polygon, >= 3 vertices */
#define COLLAGE_POLYLINE 2   /* open polyline, >= 2 vertices, drawn with half-width stroke_hw */

/* One collage: the problem statement of Sec. 3, Eq. 1 (items G, container C, initial t, r, s). */
typedef struct {
  int n_elems;                     /* >= 1 */
  const int* kind;                 /* [n_elems] COLLAGE_* */
  const int* pt_off;               /* [n_elems+1] CSR offsets (in points) into pts */
  const float* pts;                /* [2*pt_off[n_elems]] element-local x, y (unit coordinates) */
  const float* stroke_hw;          /* [n_elems] stroke half-width of polylines, world units;
                                      NULL = 0 */
  const float* params0;            /* [4*n_elems] initial (tx, ty, theta, s); s > 0 */
  const unsigned char* trainable;  /* [4*n_elems] 1 = optimise this entry; NULL = all */
  int n_rings;                     /* container: >= 1 closed rings, nonzero fill rule */
  const int* ring_off;             /* [n_rings+1] CSR offsets (in points) into ring_pts */
  const float* ring_pts;           /* [2*ring_off[n_rings]] unit coordinates */
  int grid;                        /* finest grid side in pixels; 0 = level_res[n_levels-1] */
} collage_problem;

/* Loss weights, renderer and schedule.  collage_default_options fills the paper's values:
 * alpha, beta, gamma = 3e3, 8e4, 5e-4 (Eq. 8); w_in, w_out = 1, 100 (Sec. 4.2 containment);
 * dilation widths 5 + 6k pixels (Sec. 4.2 even distribution) with weights k + 1. */
typedef struct {
  float alpha, beta, gamma, delta_down; /* Eq. 8 weights and the force weight (0 = off; < 0
                                           repels), force potential per force_kind below */
  float tau;                            /* opacity of the overlap render (Eq. 6), in (0, 1) */
  float w_in, w_out;                    /* containment penalty inside / outside (Eq. 5) */
  int n_dilations;                      /* 0..8 dilation kernels of the uniform loss (Eq. 7) */
  float dil_weight[8];
  float pad_px;                         /* padding of the overlap render, pixels, >= 0 */
  float rho_px;                         /* anti-aliasing half-width, pixels, > 0 (default 1) */
  int segs_per_cubic;                   /* line segments per cubic Bezier (default 16) */
  int n_levels;                         /* resolution pyramid (Sec. 4.3), 1..8 levels */
  int level_res[8];                     /* level sides for a problem whose grid equals
                                           level_res[n_levels-1]; others scale by
                                           grid / level_res[n_levels-1] */
  int level_iters[8];                   /* iterations per level for collage_run_schedule */
  float lr, beta1, beta2, eps;          /* Adam (default 1e-2, 0.9, 0.999, 1e-8) */
  float s_min, s_max;                   /* scale clamp after each step (default 0.05, 20) */
  int deterministic;                    /* 1: gradients reduced in a fixed order (bitwise
                                           reproducible); 0: warp-reduced float atomics */
  int tile;                             /* raster tile side 8 or 16; 0 = autotune */
  int persistent;                       /* 1: grid-stride launches sized to the SM count */
  int use_graphs;                       /* 1: collage_step replays a captured CUDA graph */
  int overlap_launches;                 /* 1: each kernel of an iteration is launched with
                                           programmatic stream serialisation, so its launch and
                                           block scheduling overlap the previous kernel's tail;
                                           results are bitwise the same either way */
  int force_kind;                       /* force term of Sec. 5 (force attraction), weight
                                           delta_down: 0 = downward, (1/wh) sum_p O(p) (1 - y_p);
                                           1 = towards the point (force_x, force_y) in unit
                                           coordinates, (1/wh) sum_p O(p) |p - (force_x, force_y)| */
  float force_x, force_y;
  int fit_controls;                     /* 1: optimise the element outlines instead of their
                                           transforms (Sec. 3, Vector Representation: closed
                                           cubic paths fitted to an item silhouette by
                                           differentiable rendering).  The parameters are then
                                           the points of every element (pts of
                                           collage_problem: cubic control points, polygon and
                                           polyline vertices) in element-local coordinates; the
                                           transforms stay at params0.  The silhouette to fit
                                           is given as the container rings (L_c of Eq. 5 with
                                           w_in = w_out is the fitting loss).  0 = off */
} collage_options;

/* Per-level sizes, for callers that allocate image buffers. */
typedef struct {
  int n_probs, n_elems, level, n_levels;
  int tile;                  /* raster tile side in use */
  long long total_pixels;    /* sum over problems of res*res at the current level */
  int pair_capacity;         /* (tile, element) pairs the bin buffers hold */
  int last_pairs;            /* pairs binned by the last iteration (after a sync) */
  int kernels_per_iter;      /* kernel launches of one collage_step iteration */
  /* How often the rarely taken kernel paths ran since collage_create (cumulative): */
  long long path_row_fallback; /* pixel rows of a (tile, element) pair that cross the outline
                                  more than 16 times, whose winding number is then taken over
                                  every segment of the outline */
  long long path_long_near;    /* emission chunks of outlines of more than 512 segments (not
                                  staged in shared memory: read from global memory per tile) */
  long long path_wide_tile;    /* tiles listing more than 32 elements (the composite ranks the
                                  list in global memory instead of by warp shuffles) */
  long long path_ring_chunk;   /* container chunks after the first 1024 segments of a ring */
} collage_info;

/* Fills *opt with the defaults listed above (one level of 1024, 50 iterations). */
void collage_default_options(collage_options* opt);

/* Validates and copies n_probs problems (n_probs > 1 is the batched form: independent collages of
 * uneven sizes run in the same launches), flattens cubic paths into segs_per_cubic line segments
 * each, allocates device memory, and selects level 0.  The current CUDA device is used.
 * Returns INVALID_ARG (with the offending field in collage_last_error(NULL)) for: n_probs < 1,
 * n_elems < 1, unknown kind, too few points, NaN/Inf or s <= 0 params, rings with < 3 points,
 * grid not divisible as the level schedule requires, tile not in {0, 8, 16}. */
collage_status collage_create(const collage_problem* probs, int n_probs,
                              const collage_options* opt, collage_t* out);

/* Selects level `level` of the pyramid: rasterises the container into I_C and W at that level's
 * resolution (Sec. 4 first paragraph, Eq. 5 mask), sizes the bin buffers, and drops captured
 * graphs.  Synchronises the device.  Params and Adam state carry over (unit coordinates). */
collage_status collage_set_level(collage_t h, int level);

/* Renders the current params (Eq. 2 and the anti-aliased rasteriser) into d_img_bw (items black
 * on white, prod(1 - c_i)) and d_img_tau (overlap render 1 - prod(1 - tau c_i^pad)); each is
 * [total_pixels] float, problems concatenated, row-major; either may be NULL.  Asynchronous. */
collage_status collage_render(collage_t h, void* stream, float* d_img_bw, float* d_img_tau);

/* One forward + backward pass at the current params: d_loss_terms [n_probs*5] receives
 * (L_c, L_o, L_u, L_force, L) per problem (Eqs. 5, 6, 7, force, 8) and d_dparams [4*n_elems] the
 * gradient dL/d(tx, ty, theta, s).  Either may be NULL.  Params are not changed.  Asynchronous. */
collage_status collage_loss_backward(collage_t h, void* stream, float* d_loss_terms,
                                     float* d_dparams);

/* n_iters >= 0 iterations of forward + backward + Adam (Eq. 4 with Adam) at the current level,
 * replaying a captured CUDA graph when use_graphs is set.  Synchronises the stream at the end to
 * check the device status; a bin overflow regrows the buffers and resumes, so exactly n_iters
 * successful iterations run.  Each iteration's Adam step is applied at the start of the next
 * iteration (inside its transform kernel); every call that reads or replaces the params
 * (get_params, get_state, set_params, step_host) applies a pending step first, so callers always
 * observe the updated params. */
collage_status collage_step(collage_t h, void* stream, int n_iters);

/* Enqueues n_iters >= 0 iterations exactly as collage_step does and returns without waiting for
 * the stream.  A bin overflow met on the device latches the status word and turns the remaining
 * enqueued iterations into no-ops (the step counter of collage_get_state counts only the ones
 * that ran); collage_sync then regrows the buffers and returns COLLAGE_ERR_OVERFLOW so that the
 * caller can enqueue the missing iterations again.  No host round trip per call: this is the
 * form for timing the device work of one iteration and for overlapping it with host work. */
collage_status collage_step_async(collage_t h, void* stream, int n_iters);

/* Runs every level of the schedule from the current one: set_level + level_iters[l] steps. */
collage_status collage_run_schedule(collage_t h, void* stream);

/* Host-buffer form of collage_step for callers without device memory: copies h_params_in
 * [4*n_elems] (NULL = keep) to the device, runs n_iters iterations, copies the params to
 * h_params_out [4*n_elems] and the last loss terms to h_loss_out [n_probs*5] (either NULL = skip)
 * and synchronises.  Pinned host memory is faster but not required; the outputs are gathered by
 * one kernel into a mapped (page-locked) staging buffer of the handle.  Unless a bin overflow has
 * to be recovered (as collage_step does), the transfers, the iterations and the status check share
 * one host round trip.  With params in, one iteration and graphs enabled, the call copies the params
 * on the host into a second mapped buffer of the handle and launches one captured graph: its
 * transform reads them from there (a pending Adam step updates the moments, the params are
 * replaced) and its last kernel writes the outputs, so no separate copy or launch precedes or
 * follows the iteration. */
collage_status collage_step_host(collage_t h, void* stream, int n_iters, const float* h_params_in,
                                 float* h_params_out, float* h_loss_out);

/* Loss terms of the most recent iteration, [n_probs*5] (device). */
collage_status collage_get_loss(collage_t h, void* stream, float* d_loss_terms);
collage_status collage_get_params(collage_t h, void* stream, float* d_params);
collage_status collage_set_params(collage_t h, void* stream, const float* d_params);

/* Outline points (fit_controls mode, and readable in any mode): d_pts [2*n_pts], the pts arrays of
 * the problems concatenated in problem order (element-local unit coordinates, CSR by pt_off).
 * get_controls reads the current points; set_controls replaces them (re-flattening every outline on
 * the device with the segs_per_cubic samples of Sec. 3 and resetting nothing else); get_control_grad
 * writes dL/d(points) of the most recent collage_loss_backward or collage_step iteration in
 * fit_controls mode (zeros before the first).  Cubic control points map to flattened vertices by
 * the Bernstein weights of their curve; polygon and polyline points are the vertices.  NULL
 * pointers return COLLAGE_ERR_INVALID_ARG; all three are asynchronous. */
collage_status collage_get_controls(collage_t h, void* stream, float* d_pts);
collage_status collage_set_controls(collage_t h, void* stream, const float* d_pts);
collage_status collage_get_control_grad(collage_t h, void* stream, float* d_dpts);

/* Skeleton-based initial positions (Sec. 4.1, Initialization): the medial axis of each problem's
 * container at the current level and its medial width, then the elements placed along the axis,
 * larger ones where the width is larger.  On the container raster (inside: coverage >= 1/2; the
 * pixels one step beyond the image are outside), D2(p) is the exact squared distance in pixels
 * from an inside pixel centre to the nearest outside pixel centre; the axis is the ridge of D2: the
 * inside pixels that are a maximum of D2 along one of the four lines through them (horizontal,
 * vertical, the two diagonals; >= both line neighbours and > one, neighbours beyond the image 0).  The elements, in decreasing
 * radius r = bin radius x s x res (pixels; ties: lower index), each take the axis pixel of largest
 * D2 (ties: lower pixel index) whose clearance min_j (|p - c_j| - r_j) over the elements already
 * placed is >= r, else the axis pixel of largest clearance (float32, fixed operation order); an
 * element's translation becomes that pixel's centre, its rotation and scale stay.  A pending Adam
 * step is applied first; the Adam state is kept.  A problem without inside pixels keeps its
 * params.  Optional outputs (device, [total_pixels] at the current level, NULL to skip):
 *   d_axis   int32 1 on the medial axis, else 0
 *   d_width  float32 medial width sqrt(D2) in pixels (0 outside the container)
 * Allocates scratch (16 B per pixel) on first use; asynchronous. */
collage_status collage_mat_init(collage_t h, void* stream, int* d_axis, float* d_width);

/* Checkpoint: d_state [12*n_elems] = params, Adam m, Adam v (device); *h_step and *h_level are
 * the Adam step count and the level.  set_state restores all of it (and sets the level). */
collage_status collage_get_state(collage_t h, void* stream, float* d_state, int* h_step,
                                 int* h_level);
collage_status collage_set_state(collage_t h, void* stream, const float* d_state, int h_step,
                                 int h_level);

/* The sorted (tile, element) bin list of the last binning: d_tile, d_elem [cap] int32; tiles are
 * numbered problem after problem, row-major within a problem; *h_n receives the pair count.
 * Synchronises the stream. */
collage_status collage_get_bins(collage_t h, void* stream, int* d_tile, int* d_elem, int cap,
                                int* h_n);

/* Device time per stage, averaged over n_iters eager iterations, into h_ms[COLLAGE_N_STAGES]
 * (see COLLAGE_STAGE_*); the kernels run on `stream`, timed with events on that stream. */
#define COLLAGE_N_STAGES 9
#define COLLAGE_STAGE_TRANSFORM 0 /* previous Adam step, transform, segment records, tile counts */
#define COLLAGE_STAGE_BIN 1       /* (empty: the transform allocates the pair slots, the emission
                                     files them in the tiles' lists) */
#define COLLAGE_STAGE_RASTER_FWD 2 /* pair emission, classification and per-pixel signed distances */
#define COLLAGE_STAGE_COMPOSITE 3 /* per-tile products and loss partials */
#define COLLAGE_STAGE_DILATE 4    /* distribution term forward and backward */
#define COLLAGE_STAGE_RASTER_BWD 5
#define COLLAGE_STAGE_REDUCE 6    /* deterministic gradient reduction */
#define COLLAGE_STAGE_LOSS 7      /* loss assembly */
#define COLLAGE_STAGE_ADAM 8      /* (empty: the Adam step is applied by the next transform) */
collage_status collage_stage_times(collage_t h, void* stream, int n_iters, float* h_ms);

/* A launch configuration of the iteration's kernels, as the autotuner chooses it. */
typedef struct {
  int tile;              /* raster tile side, 8 or 16 */
  int emit_threads;      /* threads per block of the emission / signed-distance kernel: 128, 256 */
  int chunk_px;          /* side of the emission's work items (squares of an element's tile
                            rectangle), pixels: 64 or 32 */
  float fwd_grid;        /* persistent grids of the emission, adjoint and composite kernels, as */
  float bwd_grid;        /*   multiples of (SM count x blocks resident per SM): 0.5, 1 or 2 */
  float comp_grid;
  float default_ms;      /* loss + gradient iteration time of the defaults (tile 16, 128 threads,
                            64-px chunks, grids x1), ms; 0 when the choice came from the cache */
  float best_ms;         /* iteration time of the chosen configuration, ms */
  int trials;            /* configurations timed */
  int from_cache;        /* 1: the choice of an earlier search with the same key was reused */
} collage_tuning;

/* The autotuner (no counterpart in the paper): at the current level, times the raster tile sizes
 * with the other parameters at their defaults, then in turn the emission block size, the
 * emission's chunk side and the persistent-grid multiples of the emission, adjoint and composite
 * kernels (each candidate a
 * captured one-iteration graph of loss and gradient, no Adam step, the fastest of three batches of
 * 20 replays, each timed alone from a cold L2 after a write of twice the L2 size through a
 * scratch buffer the call allocates and frees), and keeps the fastest; a launch parameter other than the tile changes only
 * when its candidate is more than 3% faster.  The choice is cached for the process, keyed on (pixels of the level, element
 * count, pair density in half-octaves, deterministic mode); a handle with the same key reuses it
 * without a search.  One configuration serves the whole handle (every problem of a batch).
 * h_best_ms (may be NULL) receives the chosen configuration's iteration time.  Params and Adam
 * state are not changed (a pending Adam step is applied as the next iteration would).
 * Synchronises the device; drops captured graphs.  On failure the previous configuration is
 * restored. */
collage_status collage_autotune(collage_t h, void* stream, float* h_best_ms);
collage_status collage_get_tuning(collage_t h, collage_tuning* out);
/* Applies a launch configuration without a search (one an earlier collage_autotune chose, saved by
 * the caller): tile, emit_threads, chunk_px and the three grid multiples must be values the
 * autotuner searches (8/16, 128/256, 64/32, 0.5/1/2); anything else returns
 * COLLAGE_ERR_INVALID_ARG and changes nothing.  The timing fields are ignored; collage_get_tuning
 * then reports zeros for them.  Synchronises the device; drops captured graphs.  On failure the
 * previous configuration is restored. */
collage_status collage_set_tuning(collage_t h, void* stream, const collage_tuning* c);

/* The even-distribution term of one res x res image, as collage_loss_backward evaluates it, and
 * its gradient with respect to the occupancy O = 1 - d_ihat, computed without allocating any
 * device memory.  The paper has no counterpart to this call.  It exists for callers that cannot
 * call cudaMalloc: code whose device memory is owned by another allocator (a framework's caching
 * allocator, a fixed arena), which a cudaMalloc behind its back would bypass, and real-time loops
 * where cudaMalloc / cudaFree, which can synchronise the device, are not acceptable.
 *   d_ihat [res*res]    items rendered black on white (the d_img_bw of collage_render), row-major
 *   d_cov  [res*res]    container coverage M_C (1 inside, 0 outside, anti-aliased at the edge)
 *   h_dil_weight [n_dilations]  host weights of the kernels of widths 5 + 6k pixels, 1..8 kernels
 *   d_loss [1]          receives L_u = sum_k w_k sum_p M_C (1 - O) (1 - min(1, box_k(O)))
 *   d_grad_occ [res*res] receives dL_u/dO
 * Scratch lives in a file-scope device array sized for COLLAGE_NOALLOC_MAX_PIXELS pixels (about
 * 5 MiB, held by every GPU that loads the library until the process exits).  res*res above that
 * maximum, res < 1, n_dilations outside 1..8 or a NULL pointer return COLLAGE_ERR_INVALID_ARG
 * before any device work; CUDA failures return COLLAGE_ERR_CUDA.  The first call on a device looks
 * up the array's device address and sets the dilation kernels' shared-memory limit (once per
 * device, with that device current); make that first call before any stream capture.  All calls share the one array and it keeps the last call's
 * contents, so calls that overlap on the GPU (different streams, threads or devices sharing a
 * context) race: serialise them.  Asynchronous on `stream`; inputs must stay valid until it runs. */
#define COLLAGE_NOALLOC_MAX_PIXELS (1024 * 1024)
collage_status collage_uniform_term_noalloc(void* stream, int res, int n_dilations,
                                            const float* h_dil_weight, const float* d_ihat,
                                            const float* d_cov, float* d_loss, float* d_grad_occ);

/* Quality metrics of the collage at the current params (Sec. 6, "Metrics of Collage Quality";
 * the layout non-uniformity of the uniformity ablation, Sec. 6.1), from a render pass at the
 * current level.  A pixel is object where O = 1 - Ihat >= 1/2, shape where the container coverage
 * is >= 1/2, and overlap where at least two elements have sd >= 0.  h_metrics (host memory,
 * [n_probs * 8] doubles) receives per problem: object pixels inside the shape, shape pixels,
 * overlap pixels, object pixels outside the shape, then LC = inside / shape, OO = overlap /
 * shape, EA = outside / shape, and L-nU = the mean over the non-object shape pixels of the
 * squared distance (unit coordinates) to the nearest object pixel centre (0 when there is no
 * object pixel or no such pixel).  Applies a pending Adam step first; synchronises `stream`;
 * allocates its scratch on the first call at a level size. */
collage_status collage_metrics(collage_t h, void* stream, double* h_metrics);

/* Measurement helper, no counterpart in the paper: the FP32 FMA rate of the current device in
 * TFLOP/s (eight independent FMA chains per thread at full occupancy, best of three timed launches
 * after a warm-up), the ceiling of the ALU-bound distance kernel.  Writes *h_tflops (host memory);
 * INVALID_ARG for NULL, CUDA on a launch or event failure.  Synchronises `stream`. */
collage_status collage_fp32_peak(void* stream, float* h_tflops);

/* Sizes of the current level and the path counters above.  Synchronises the device. */
collage_status collage_get_info(collage_t h, collage_info* out);
/* Waits for the stream and returns any latched device error. */
collage_status collage_sync(collage_t h, void* stream);
/* Message of the last error on h (h = NULL: the last collage_create failure of this thread). */
const char* collage_last_error(collage_t h);
void collage_destroy(collage_t h);

#ifdef __cplusplus
}
#endif
#endif /* COLLAGE_H */
