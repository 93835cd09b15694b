/* FP64 CPU oracle of the image-space collage hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use this code.  It shares
 * no source, header, table or helper with the CUDA library, and the library never calls it.
 *
 * What it computes (Wang & Lu, "Image-Space Collage and Packing with Differentiable Rendering"):
 *   - element outlines: closed paths of cubic Beziers (Sec. 3 "Vector Representation"),
 *     flattened here at uniform parameter steps, or polygons / open polylines;
 *   - the per-element similarity transform P' = r (P (.) s) + t (Eq. 2);
 *   - anti-aliased coverage of every pixel from winding number and signed distance, the
 *     differentiable rasteriser the method relies on (Sec. 3 "Differentiable Rendering");
 *   - the container target image I_C and penalty mask W (Sec. 4, text before Eq. 5);
 *   - containment (Eq. 5), non-overlap (Eq. 6), even-distribution (Eq. 7) and downward-force
 *     (Sec. 5 "Force Attraction") losses, summed with the weights of Eq. 8;
 *   - the gradient of that loss with respect to (t, theta, s) by two independent routes;
 *   - the Adam update that replaces plain gradient descent of Eq. 4;
 *   - the tile-bin list of the library's binning rule (a combinatorial specification).
 * Every reading of an ambiguous passage is listed where it is used in collage_oracle.c.
 *
 * Everything is double precision; float inputs are promoted exactly.
 *
 * Parity status: every function here is pinned by closed forms, brute force or finite differences
 * in tests/test_oracle_pins.py, except the multi-iteration optimisation trajectory (which the
 * tests compare only over one Adam step): trajectory parity unpinned beyond one step.
 */
#ifndef COLLAGE_ORACLE_H
#define COLLAGE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ora_scene ora_scene;

typedef struct {
  double alpha, beta, gamma, delta; /* Eq. 8 weights, plus the force weight */
  double tau;                       /* fixed opacity of the overlap render (Eq. 6) */
  double w_in, w_out;               /* penalty mask values inside / outside (Eq. 5) */
  int n_dil;                        /* number of dilation kernels (Eq. 7) */
  double dil_weight[8];             /* weight of each dilation kernel */
  double pad_px;                    /* padding offset in pixels (overlap render only) */
  double rho_px;                    /* anti-aliasing filter half-width in pixels */
  int cull;                         /* 1: skip elements whose grown bounding box misses the pixel */
  int force_kind;                   /* 0: downward, potential 1 - y; 1: towards the point
                                       (force_x, force_y), potential |p - (force_x, force_y)| */
  double force_x, force_y;          /* the force point, unit coordinates */
} ora_opts;

/* Scene: element outlines (flattened once) and the container rings.  Inputs are copied. */
ora_scene* ora_scene_create(int n, const int* kind, const int* pt_off, const float* pts,
                            const float* hw, int segs_per_cubic, int n_rings,
                            const int* ring_off, const float* ring_pts);
void ora_scene_free(ora_scene* sc);
int ora_n_vertices(const ora_scene* sc, int e);
int ora_total_vertices(const ora_scene* sc);
void ora_local_vertices(const ora_scene* sc, int e, double* out_xy);
void ora_world_vertices(const ora_scene* sc, const double* params, int e, double* out_xy);

/* Signed distance of element e at world points xy[2*npts] (unit coordinates): positive inside.
 * Also returns the index of the closest segment and its clamped parameter (either may be NULL). */
void ora_signed_distance(const ora_scene* sc, const double* params, int e, int npts,
                         const double* xy, double* sd, int* seg, double* u);
void ora_container_sd(const ora_scene* sc, int npts, const double* xy, double* sd);

/* Images on a res x res grid, row-major, any output may be NULL:
 * ihat = prod(1 - c_i), atau = 1 - prod(1 - tau c_i^pad), covc = container coverage. */
void ora_render(const ora_scene* sc, const double* params, int res, const ora_opts* o,
                double* ihat, double* atau, double* covc);

/* Loss terms [L_c, L_o, L_u, L_down, L] and, if requested, the gradient dL/d(tx,ty,theta,s):
 * grad_a through per-vertex gradients and the Jacobian of Eq. 2 (grad_v receives the per-vertex
 * world gradients, 2 per flattened vertex), grad_b through the spatial gradient of the signed
 * distance.  Any output may be NULL. */
void ora_eval(const ora_scene* sc, const double* params, int res, const ora_opts* o,
              double* terms, double* grad_a, double* grad_b, double* grad_v);

/* The even-distribution term of Eq. 7 alone, on one res x res image: occ = O = 1 - Ihat and covc
 * the container coverage (row-major, res*res each), K kernels of widths 5 + 6k px with weights
 * w[K].  *Lu receives L_u; gou (may be NULL) receives dL_u/dO per pixel.  ora_eval uses it. */
void ora_uniform_term(int res, int K, const double* w, const double* occ, const double* covc,
                      double* Lu, double* gou);

/* One Adam step (bias-corrected, step >= 1) on params[4n]; entries whose trainable flag is 0 are
 * left unchanged, s is clamped to [s_min, s_max] after the step. */
void ora_adam(int n, double* p, double* m, double* v, const double* g, int step, double lr,
              double b1, double b2, double eps, const unsigned char* trainable, double s_min,
              double s_max);

/* Tile bins of the binning rule, sorted by (tile, element); returns the pair count (writes at
 * most cap pairs).  Tiles are numbered row-major, tile x fastest. */
long ora_bins(const ora_scene* sc, const float* params, int res, int tile, float rho_px,
              float pad_px, int* tile_out, int* elem_out, long cap);
/* The same tile set by brute force over all (element, tile) pairs. */
long ora_bins_bruteforce(const ora_scene* sc, const float* params, int res, int tile,
                         float rho_px, float pad_px, int* tile_out, int* elem_out, long cap);
float ora_bin_radius(const ora_scene* sc, int e);

/* Algorithmic work: sum over elements of (pixel centres inside the element's world bounding box
 * grown by rho + pad (+ stroke half-width)) x (segments of the element). */
double ora_pair_work(const ora_scene* sc, const double* params, int res, const ora_opts* o);

/* Quality metrics of the render at params on the R x R grid (Sec. 6, "Metrics of Collage
 * Quality", and the layout non-uniformity of the uniformity ablation, Sec. 6.1).  A pixel is
 * object where O = 1 - Ihat >= 1/2, shape where the container coverage is >= 1/2, and overlap
 * where at least two elements have sd >= 0 (c_i >= 1/2).  out[8]:
 *   [0] object pixels inside the shape, [1] shape pixels, [2] overlap pixels,
 *   [3] object pixels outside the shape,
 *   [4] LC = [0]/[1], [5] OO = [2]/[1], [6] EA = [3]/[1], [7] 0.
 * obj_out [R*R] (may be NULL) receives the object mask (1: object) and shape_out [R*R] (may be
 * NULL) the shape mask; the layout non-uniformity L-nU (the mean over the non-object shape pixels
 * of the squared distance, unit coordinates, from the pixel centre to the nearest object pixel
 * centre) is formed from them by oracle.py, as a nearest-neighbour search over every object
 * pixel. */
void ora_metrics(const ora_scene* sc, const double* params, int R, const ora_opts* o, double* out,
                 unsigned char* obj_out, unsigned char* shape_out);

/* Threads the OpenMP loops use from now on (n < 1: all the host's cores); returns the previous
 * setting.  For timing the oracle on one core. */
int ora_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
