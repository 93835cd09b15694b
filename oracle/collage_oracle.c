/* FP64 CPU oracle of the image-space collage hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow restatement of the method of Wang & Lu (SIGGRAPH Conf. Papers 2025, arXiv
 * 2406.04008), used to check the CUDA library.  It shares no code with that library.
 * Loops run over every pixel and every element; the only shortcut is the exact cull described at
 * element_bbox(), which tests check against the uncull'd result.
 *
 * Conventions (readings of passages the paper leaves open):
 *  - unit-square world coordinates, y pointing down; pixel (i, j) has its centre at
 *    ((j + 1/2)/R, (i + 1/2)/R) on an R x R grid;
 *  - coverage c = S(sd / rho) with S(x) = 1/2 + 3x/4 - x^3/4 on [-1, 1] (0 below, 1 above),
 *    sd the signed distance (positive inside), rho = rho_px / R; S is C^1 and odd about 1/2, so
 *    it preserves area across a straight edge, and it is exactly 0 / 1 beyond +-rho;
 *  - closed outlines use the nonzero winding rule with a +x ray and the half-open crossing test;
 *    an open polyline of half-width hw (world units, not scaled by s) has sd = hw - d;
 *  - items render black on white: Ihat = prod_i (1 - c_i) (Sec. 4, text before Eq. 5);
 *  - padding offsets each item outward by pad_px pixels in the overlap render only;
 *  - Eq. 6's indicator has no useful gradient, so the overlap term is the surrogate
 *    max(0, A_tau - tau) with A_tau = 1 - prod_i (1 - tau c_i^pad), tau = 1/2 by default;
 *  - Eq. 7: K box kernels of widths 5 + 6k pixels (k = 0..K-1), D_k = min(1, box sum of O),
 *    L_u = sum_k w_k sum_p M_C(p) (1 - O(p)) (1 - D_k(p)), unnormalised, zero padding;
 *  - force terms (Sec. 5, force attraction): L_f = (1/wh) sum_p O(p) phi(p) with the potential
 *    phi = 1 - y (downward) or phi = |p - c| (towards a point c; a negative weight repels);
 *  - W = w_in where the container coverage is >= 1/2, else w_out;
 *  - one-sided derivatives at kinks: d max(0,x)/dx = 0 and d min(1,B)/dB = 0 at the kink, and
 *    the first closest segment (lowest index) wins ties.
 */
#include "collage_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double x, y;
} vec2;

struct ora_scene {
  int n;
  int* kind;    /* 0 cubic path (closed), 1 polygon (closed), 2 polyline (open) */
  int* voff;    /* [n+1] offsets into vloc */
  vec2* vloc;   /* flattened element-local vertices */
  double* hw;   /* stroke half-width of open polylines, world units */
  float* rbin;  /* bin radius: largest |control point|, rounded to float */
  int nr;
  int* roff;
  vec2* rpts;   /* container rings, unit coordinates */
};

/* ---------------------------------------------------------------------------------------------
 * Anti-aliasing filter (reading of the renderer of Sec. 3 "Differentiable Rendering")
 * ------------------------------------------------------------------------------------------- */
static double S(double x) {
  if (x <= -1.0) return 0.0;
  if (x >= 1.0) return 1.0;
  return 0.5 + 0.75 * x - 0.25 * x * x * x;
}
static double dS(double x) {
  if (x <= -1.0 || x >= 1.0) return 0.0;
  return 0.75 * (1.0 - x * x);
}

static int is_closed(int kind) { return kind != 2; }
static int n_verts(const ora_scene* sc, int e) { return sc->voff[e + 1] - sc->voff[e]; }
static int n_segs(const ora_scene* sc, int e) {
  int nv = n_verts(sc, e);
  return is_closed(sc->kind[e]) ? nv : nv - 1;
}

/* ---------------------------------------------------------------------------------------------
 * Scene construction: flattening of cubic Bezier paths (Sec. 3 "Vector Representation")
 * A closed path of N cubics has 3N control points; curve k runs through control points
 * 3k, 3k+1, 3k+2 and 3k+3 (mod 3N).  Each curve is sampled at t = j / segs, j = 0..segs-1, with the
 * Bernstein form; consecutive samples (and the last to the first) are joined by segments.
 * ------------------------------------------------------------------------------------------- */
ora_scene* ora_scene_create(int n, const int* kind, const int* pt_off, const float* pts,
                            const float* hw, int segs_per_cubic, int n_rings,
                            const int* ring_off, const float* ring_pts) {
  ora_scene* sc = (ora_scene*)calloc(1, sizeof(ora_scene));
  sc->n = n;
  sc->kind = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  sc->voff = (int*)malloc(sizeof(int) * (n + 1));
  sc->hw = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  sc->rbin = (float*)malloc(sizeof(float) * (n > 0 ? n : 1));
  int total = 0;
  for (int e = 0; e < n; ++e) {
    int np = pt_off[e + 1] - pt_off[e];
    total += kind[e] == 0 ? (np / 3) * segs_per_cubic : np;
  }
  sc->vloc = (vec2*)malloc(sizeof(vec2) * (total > 0 ? total : 1));
  int w = 0;
  for (int e = 0; e < n; ++e) {
    const float* p = pts + 2 * pt_off[e];
    int np = pt_off[e + 1] - pt_off[e];
    sc->kind[e] = kind[e];
    sc->hw[e] = (kind[e] == 2 && hw) ? (double)hw[e] : 0.0;
    sc->voff[e] = w;
    double rmax = 0.0;
    for (int k = 0; k < np; ++k) {
      double x = p[2 * k], y = p[2 * k + 1];
      double r = sqrt(x * x + y * y);
      if (r > rmax) rmax = r;
    }
    sc->rbin[e] = (float)rmax;
    if (kind[e] == 0) {
      int ncub = np / 3;
      for (int k = 0; k < ncub; ++k) {
        const float* P0 = p + 2 * (3 * k);
        const float* P1 = p + 2 * (3 * k + 1);
        const float* P2 = p + 2 * (3 * k + 2);
        const float* P3 = p + 2 * ((3 * k + 3) % np);
        for (int j = 0; j < segs_per_cubic; ++j) {
          double t = (double)j / (double)segs_per_cubic, s = 1.0 - t;
          double b0 = s * s * s, b1 = 3.0 * s * s * t, b2 = 3.0 * s * t * t, b3 = t * t * t;
          sc->vloc[w].x = b0 * P0[0] + b1 * P1[0] + b2 * P2[0] + b3 * P3[0];
          sc->vloc[w].y = b0 * P0[1] + b1 * P1[1] + b2 * P2[1] + b3 * P3[1];
          ++w;
        }
      }
    } else {
      for (int k = 0; k < np; ++k) {
        sc->vloc[w].x = p[2 * k];
        sc->vloc[w].y = p[2 * k + 1];
        ++w;
      }
    }
  }
  sc->voff[n] = w;
  sc->nr = n_rings;
  sc->roff = (int*)malloc(sizeof(int) * (n_rings + 1));
  int nrp = ring_off[n_rings];
  sc->rpts = (vec2*)malloc(sizeof(vec2) * (nrp > 0 ? nrp : 1));
  for (int r = 0; r <= n_rings; ++r) sc->roff[r] = ring_off[r];
  for (int k = 0; k < nrp; ++k) {
    sc->rpts[k].x = ring_pts[2 * k];
    sc->rpts[k].y = ring_pts[2 * k + 1];
  }
  return sc;
}

void ora_scene_free(ora_scene* sc) {
  if (!sc) return;
  free(sc->kind);
  free(sc->voff);
  free(sc->vloc);
  free(sc->hw);
  free(sc->rbin);
  free(sc->roff);
  free(sc->rpts);
  free(sc);
}

int ora_n_vertices(const ora_scene* sc, int e) { return n_verts(sc, e); }
int ora_total_vertices(const ora_scene* sc) { return sc->voff[sc->n]; }
float ora_bin_radius(const ora_scene* sc, int e) { return sc->rbin[e]; }

void ora_local_vertices(const ora_scene* sc, int e, double* out) {
  for (int k = 0; k < n_verts(sc, e); ++k) {
    out[2 * k] = sc->vloc[sc->voff[e] + k].x;
    out[2 * k + 1] = sc->vloc[sc->voff[e] + k].y;
  }
}

/* Eq. 2: P' = r (P (.) s) + t with r the rotation by theta and s a uniform scale. */
static vec2 transform(const double* q, vec2 v) {
  double c = cos(q[2]), sn = sin(q[2]), s = q[3];
  vec2 o;
  o.x = c * (s * v.x) - sn * (s * v.y) + q[0];
  o.y = sn * (s * v.x) + c * (s * v.y) + q[1];
  return o;
}

void ora_world_vertices(const ora_scene* sc, const double* params, int e, double* out) {
  for (int k = 0; k < n_verts(sc, e); ++k) {
    vec2 w = transform(params + 4 * e, sc->vloc[sc->voff[e] + k]);
    out[2 * k] = w.x;
    out[2 * k + 1] = w.y;
  }
}

/* ---------------------------------------------------------------------------------------------
 * Distance and winding of a point against a chain of segments
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  double d;    /* distance to the closest segment */
  int seg;     /* index of the first closest segment */
  double u;    /* clamped parameter of the closest point on it */
  int wind;    /* nonzero winding number (closed chains) */
} chain_query;

/* Closest point on segment a-b: q = a + u (b - a), u = clamp(((p-a).(b-a)) / |b-a|^2, 0, 1).
 * Winding: a segment crosses the +x ray from p when (a.y <= p.y) != (b.y <= p.y) and the crossing
 * lies strictly right of p; upward crossings count +1, downward -1. */
static void chain_accumulate(vec2 p, vec2 a, vec2 b, int idx, int closed, chain_query* cq) {
  double ex = b.x - a.x, ey = b.y - a.y;
  double wx = p.x - a.x, wy = p.y - a.y;
  double ee = ex * ex + ey * ey;
  double u = ee > 0.0 ? (wx * ex + wy * ey) / ee : 0.0;
  if (u < 0.0) u = 0.0;
  if (u > 1.0) u = 1.0;
  double qx = wx - u * ex, qy = wy - u * ey;
  double d = sqrt(qx * qx + qy * qy);
  if (d < cq->d) {
    cq->d = d;
    cq->seg = idx;
    cq->u = u;
  }
  if (closed) {
    double cross = ex * wy - ey * wx; /* > 0: crossing right of p for an upward segment */
    if (a.y <= p.y) {
      if (b.y > p.y && cross > 0.0) cq->wind += 1;
    } else {
      if (b.y <= p.y && cross < 0.0) cq->wind -= 1;
    }
  }
}

/* Element query with world vertices wv of element e. */
static chain_query element_query(const ora_scene* sc, int e, const vec2* wv, vec2 p) {
  chain_query cq = {INFINITY, -1, 0.0, 0};
  int nv = n_verts(sc, e), closed = is_closed(sc->kind[e]);
  int ns = closed ? nv : nv - 1;
  for (int j = 0; j < ns; ++j) chain_accumulate(p, wv[j], wv[(j + 1) % nv], j, closed, &cq);
  return cq;
}

static double element_sd(const ora_scene* sc, int e, const chain_query* cq) {
  if (is_closed(sc->kind[e])) return cq->wind != 0 ? cq->d : -cq->d;
  return sc->hw[e] - cq->d;
}

void ora_signed_distance(const ora_scene* sc, const double* params, int e, int npts,
                         const double* xy, double* sd, int* seg, double* u) {
  int nv = n_verts(sc, e);
  vec2* wv = (vec2*)malloc(sizeof(vec2) * (nv > 0 ? nv : 1));
  for (int k = 0; k < nv; ++k) wv[k] = transform(params + 4 * e, sc->vloc[sc->voff[e] + k]);
  for (int i = 0; i < npts; ++i) {
    vec2 p = {xy[2 * i], xy[2 * i + 1]};
    chain_query cq = element_query(sc, e, wv, p);
    sd[i] = element_sd(sc, e, &cq);
    if (seg) seg[i] = cq.seg;
    if (u) u[i] = cq.u;
  }
  free(wv);
}

/* Container: all rings together under the nonzero rule. */
static double container_sd_at(const ora_scene* sc, vec2 p) {
  chain_query cq = {INFINITY, -1, 0.0, 0};
  for (int r = 0; r < sc->nr; ++r) {
    int b = sc->roff[r], nv = sc->roff[r + 1] - b;
    for (int j = 0; j < nv; ++j)
      chain_accumulate(p, sc->rpts[b + j], sc->rpts[b + (j + 1) % nv], j, 1, &cq);
  }
  return cq.wind != 0 ? cq.d : -cq.d;
}

void ora_container_sd(const ora_scene* sc, int npts, const double* xy, double* sd) {
  for (int i = 0; i < npts; ++i) {
    vec2 p = {xy[2 * i], xy[2 * i + 1]};
    sd[i] = container_sd_at(sc, p);
  }
}

/* ---------------------------------------------------------------------------------------------
 * Per-evaluation geometry: world vertices and grown bounding boxes.
 * The cull is exact: outside the bounding box grown by m = rho + pad (+ hw for strokes) every
 * point is farther than m from the outline and outside it, so c = c^pad = 0 and dS = 0 there.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  vec2* wv;       /* world vertices, all elements, indexed like vloc */
  double* box;    /* [4n] xmin, ymin, xmax, ymax grown by the margin */
} world_geom;

static world_geom make_world(const ora_scene* sc, const double* params, double rho, double pad) {
  world_geom g;
  int V = sc->voff[sc->n];
  g.wv = (vec2*)malloc(sizeof(vec2) * (V > 0 ? V : 1));
  g.box = (double*)malloc(sizeof(double) * 4 * (sc->n > 0 ? sc->n : 1));
  for (int e = 0; e < sc->n; ++e) {
    double x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
    for (int k = sc->voff[e]; k < sc->voff[e + 1]; ++k) {
      g.wv[k] = transform(params + 4 * e, sc->vloc[k]);
      if (g.wv[k].x < x0) x0 = g.wv[k].x;
      if (g.wv[k].x > x1) x1 = g.wv[k].x;
      if (g.wv[k].y < y0) y0 = g.wv[k].y;
      if (g.wv[k].y > y1) y1 = g.wv[k].y;
    }
    double m = rho + pad + (is_closed(sc->kind[e]) ? 0.0 : sc->hw[e]);
    g.box[4 * e] = x0 - m;
    g.box[4 * e + 1] = y0 - m;
    g.box[4 * e + 2] = x1 + m;
    g.box[4 * e + 3] = y1 + m;
  }
  return g;
}

static void free_world(world_geom* g) {
  free(g->wv);
  free(g->box);
}

static int culled(const world_geom* g, int e, vec2 p) {
  const double* b = g->box + 4 * e;
  return p.x < b[0] || p.x > b[2] || p.y < b[1] || p.y > b[3];
}

static vec2 pixel_centre(int i, int j, int R) {
  vec2 p = {((double)j + 0.5) / (double)R, ((double)i + 0.5) / (double)R};
  return p;
}

/* ---------------------------------------------------------------------------------------------
 * Rendering (Sec. 4 first paragraph): Ihat, the overlap composite, and the container target
 * ------------------------------------------------------------------------------------------- */
static void container_images(const ora_scene* sc, int R, double rho, double* covc) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < R; ++j) covc[(long)i * R + j] = S(container_sd_at(sc, pixel_centre(i, j, R)) / rho);
}

static void render_items(const ora_scene* sc, const world_geom* g, int R, double rho, double pad,
                         double tau, int cull, double* ihat, double* atau) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < R; ++i) {
    for (int j = 0; j < R; ++j) {
      vec2 p = pixel_centre(i, j, R);
      double keep = 1.0, keep_tau = 1.0;
      for (int e = 0; e < sc->n; ++e) {
        if (cull && culled(g, e, p)) continue;
        chain_query cq = element_query(sc, e, g->wv + sc->voff[e], p);
        double sd = element_sd(sc, e, &cq);
        double c = S(sd / rho), cp = S((sd + pad) / rho);
        keep *= 1.0 - c;
        keep_tau *= 1.0 - tau * cp;
      }
      if (ihat) ihat[(long)i * R + j] = keep;
      if (atau) atau[(long)i * R + j] = 1.0 - keep_tau;
    }
  }
}

void ora_render(const ora_scene* sc, const double* params, int R, const ora_opts* o,
                double* ihat, double* atau, double* covc) {
  double rho = o->rho_px / R, pad = o->pad_px / R;
  if (covc) container_images(sc, R, rho, covc);
  if (ihat || atau) {
    world_geom g = make_world(sc, params, rho, pad);
    render_items(sc, &g, R, rho, pad, o->tau, o->cull, ihat, atau);
    free_world(&g);
  }
}

/* ---------------------------------------------------------------------------------------------
 * Even-distribution term (Eq. 7): box sums of the occupancy with zero padding.
 * ------------------------------------------------------------------------------------------- */
static double box_sum(const double* img, int R, int i, int j, int r) {
  double s = 0.0;
  for (int di = -r; di <= r; ++di) {
    int ii = i + di;
    if (ii < 0 || ii >= R) continue;
    for (int dj = -r; dj <= r; ++dj) {
      int jj = j + dj;
      if (jj < 0 || jj >= R) continue;
      s += img[(long)ii * R + jj];
    }
  }
  return s;
}

/* Eq. 7 over one R x R image, in the reading of the header: for k = 0..K-1 the box of width
 * 5 + 6k px, B_k = its zero-padded sum of the occupancy O, D_k = min(1, B_k), and
 *   L_u = sum_k w_k sum_p M(p) (1 - O(p)) (1 - D_k(p)),
 * with M the container coverage.  Its derivative in O(q), by the chain rule through the min
 * (one-sided at the kink: d min(1, B)/dB = 0 at B = 1):
 *   dL_u/dO(q) = sum_k w_k [ -M(q)(1 - D_k(q)) - sum_{p in box_k(q)} M(p)(1 - O(p)) 1[B_k(p) < 1] ]
 * (the box is symmetric, so q in box_k(p) is p in box_k(q)).  gou may be NULL. */
void ora_uniform_term(int R, int K, const double* w, const double* occ, const double* covc,
                      double* Lu, double* gou) {
  const long NP = (long)R * R;
  double* bsum = (double*)malloc(sizeof(double) * NP * (K > 0 ? K : 1));
  double* rowsum = (double*)malloc(sizeof(double) * (R > 0 ? R : 1));
  double total = 0.0;
  for (int k = 0; k < K; ++k) {
    int r = (5 + 6 * k - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < R; ++i) {
      rowsum[i] = 0.0;
      for (int j = 0; j < R; ++j) {
        long p = (long)i * R + j;
        double B = box_sum(occ, R, i, j, r);
        bsum[k * NP + p] = B;
        double D = B < 1.0 ? B : 1.0;
        rowsum[i] += covc[p] * (1.0 - occ[p]) * (1.0 - D);
      }
    }
    double lk = 0.0; /* rows summed in order: the result does not depend on the thread count */
    for (int i = 0; i < R; ++i) lk += rowsum[i];
    total += w[k] * lk;
  }
  free(rowsum);
  *Lu = total;
  if (gou) {
    double* G = (double*)malloc(sizeof(double) * (NP > 0 ? NP : 1));
    for (long p = 0; p < NP; ++p) gou[p] = 0.0;
    for (int k = 0; k < K; ++k) {
      int r = (5 + 6 * k - 1) / 2;
      for (long p = 0; p < NP; ++p) {
        double B = bsum[k * NP + p];
        G[p] = B < 1.0 ? covc[p] * (1.0 - occ[p]) : 0.0;
      }
#pragma omp parallel for schedule(static)
      for (int i = 0; i < R; ++i)
        for (int j = 0; j < R; ++j) {
          long p = (long)i * R + j;
          double B = bsum[k * NP + p], D = B < 1.0 ? B : 1.0;
          gou[p] += w[k] * (-covc[p] * (1.0 - D) - box_sum(G, R, i, j, r));
        }
    }
    free(G);
  }
  free(bsum);
}

/* ---------------------------------------------------------------------------------------------
 * Loss (Eqs. 5-8) and gradient
 * ------------------------------------------------------------------------------------------- */
/* Potential of the force term at pixel centre (x, y) (unit coordinates). */
static double force_potential(const ora_opts* o, double x, double y) {
  if (o->force_kind == 1) return hypot(x - o->force_x, y - o->force_y);
  return 1.0 - y;
}

void ora_eval(const ora_scene* sc, const double* params, int R, const ora_opts* o, double* terms,
              double* grad_a, double* grad_b, double* grad_v) {
  const long NP = (long)R * R;
  const double rho = o->rho_px / R, pad = o->pad_px / R, tau = o->tau, inv_wh = 1.0 / (double)NP;
  world_geom g = make_world(sc, params, rho, pad);
  double* covc = (double*)malloc(sizeof(double) * NP);
  double* ihat = (double*)malloc(sizeof(double) * NP);
  double* atau = (double*)malloc(sizeof(double) * NP);
  double* occ = (double*)malloc(sizeof(double) * NP);
  container_images(sc, R, rho, covc);
  render_items(sc, &g, R, rho, pad, tau, o->cull, ihat, atau);
  for (long p = 0; p < NP; ++p) occ[p] = 1.0 - ihat[p];

  /* Eq. 5 (containment, W-weighted squared difference), Eq. 6 surrogate, force, Eq. 7 */
  double Lc = 0.0, Lo = 0.0, Ld = 0.0, Lu = 0.0;
  for (int i = 0; i < R; ++i) {
    double y = ((double)i + 0.5) / (double)R;
    for (int j = 0; j < R; ++j) {
      long p = (long)i * R + j;
      double x = ((double)j + 0.5) / (double)R;
      double ic = 1.0 - covc[p];
      double w = covc[p] >= 0.5 ? o->w_in : o->w_out;
      Lc += w * (ihat[p] - ic) * (ihat[p] - ic);
      Lo += atau[p] > tau ? atau[p] - tau : 0.0;
      Ld += occ[p] * force_potential(o, x, y);
    }
  }
  Lc *= inv_wh;
  Lo *= inv_wh;
  Ld *= inv_wh;

  const int want_grad = grad_a || grad_b || grad_v;
  double* gou = want_grad ? (double*)calloc(NP, sizeof(double)) : NULL;
  ora_uniform_term(R, o->n_dil, o->dil_weight, occ, covc, &Lu, gou);
  double L = o->alpha * Lc + o->beta * Lo + o->gamma * Lu + o->delta * Ld;
  if (terms) {
    terms[0] = Lc;
    terms[1] = Lo;
    terms[2] = Lu;
    terms[3] = Ld;
    terms[4] = L;
  }

  if (want_grad) {
    /* Per-pixel adjoints of Ihat and A_tau */
    double* gI = (double*)malloc(sizeof(double) * NP);
    double* gA = (double*)malloc(sizeof(double) * NP);
    for (int i = 0; i < R; ++i) {
      double y = ((double)i + 0.5) / (double)R;
      for (int j = 0; j < R; ++j) {
        long p = (long)i * R + j;
        double x = ((double)j + 0.5) / (double)R;
        double ic = 1.0 - covc[p];
        double w = covc[p] >= 0.5 ? o->w_in : o->w_out;
        /* O = 1 - Ihat, so the O-terms enter with a minus sign */
        gI[p] = o->alpha * inv_wh * 2.0 * w * (ihat[p] - ic) - o->gamma * gou[p] -
                o->delta * inv_wh * force_potential(o, x, y);
        gA[p] = atau[p] > tau ? o->beta * inv_wh : 0.0;
      }
    }

    int V = sc->voff[sc->n], n = sc->n;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double* acc_v = (double*)calloc((size_t)nth * 2 * (V > 0 ? V : 1), sizeof(double));
    double* acc_b = (double*)calloc((size_t)nth * 4 * (n > 0 ? n : 1), sizeof(double));
#pragma omp parallel
    {
      int tid = 0;
#ifdef _OPENMP
      tid = omp_get_thread_num();
#endif
      double* gv = acc_v + (size_t)tid * 2 * V;
      double* gb = acc_b + (size_t)tid * 4 * n;
      int* list = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
      chain_query* qs = (chain_query*)malloc(sizeof(chain_query) * (n > 0 ? n : 1));
      double* cs = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
      double* cps = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
      double* sds = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
#pragma omp for schedule(static)
      for (int i = 0; i < R; ++i) {
        for (int j = 0; j < R; ++j) {
          long pix = (long)i * R + j;
          vec2 p = pixel_centre(i, j, R);
          int m = 0;
          for (int e = 0; e < n; ++e) {
            if (o->cull && culled(&g, e, p)) continue;
            list[m] = e;
            qs[m] = element_query(sc, e, g.wv + sc->voff[e], p);
            sds[m] = element_sd(sc, e, &qs[m]);
            cs[m] = S(sds[m] / rho);
            cps[m] = S((sds[m] + pad) / rho);
            ++m;
          }
          for (int a = 0; a < m; ++a) {
            int e = list[a];
            double others = 1.0, others_tau = 1.0;
            for (int b = 0; b < m; ++b) {
              if (b == a) continue;
              others *= 1.0 - cs[b];
              others_tau *= 1.0 - tau * cps[b];
            }
            /* dIhat/dc_e = -prod_{f != e}(1 - c_f);  dA/dc^pad_e = tau prod_{f != e}(1 - tau c^pad_f) */
            double gsd = gI[pix] * (-others) * dS(sds[a] / rho) / rho +
                         gA[pix] * tau * others_tau * dS((sds[a] + pad) / rho) / rho;
            if (gsd == 0.0 || qs[a].d == 0.0) continue;
            /* closest segment a-b, closest point q, unit normal nrm from q towards p */
            int nv = n_verts(sc, e);
            const vec2* wv = g.wv + sc->voff[e];
            int j0 = qs[a].seg, j1 = (j0 + 1) % nv;
            double u = qs[a].u;
            vec2 A = wv[j0], Bv = wv[j1];
            double qx = A.x + u * (Bv.x - A.x), qy = A.y + u * (Bv.y - A.y);
            double nx = (p.x - qx) / qs[a].d, ny = (p.y - qy) / qs[a].d;
            /* sd = +-d (closed, sign of the winding) or hw - d (open) */
            double sgn = is_closed(sc->kind[e]) ? (qs[a].wind != 0 ? 1.0 : -1.0) : -1.0;
            /* route A: d(d)/dA = -n (1-u), d(d)/dB = -n u */
            double* gva = gv + 2 * (sc->voff[e] + j0);
            double* gvb = gv + 2 * (sc->voff[e] + j1);
            gva[0] += gsd * sgn * (-nx) * (1.0 - u);
            gva[1] += gsd * sgn * (-ny) * (1.0 - u);
            gvb[0] += gsd * sgn * (-nx) * u;
            gvb[1] += gsd * sgn * (-ny) * u;
            /* route B: spatial gradient of sd at p, nabla_p sd = sgn * n */
            const double* q = params + 4 * e;
            double gx = sgn * nx, gy = sgn * ny;
            double rx = p.x - q[0], ry = p.y - q[1];
            double dsd_dth = -(gx * (-ry) + gy * rx); /* -grad . J (p - t), J = [[0,-1],[1,0]] */
            double dsd_ds;
            if (is_closed(sc->kind[e]))
              dsd_ds = (sds[a] - (gx * rx + gy * ry)) / q[3];
            else /* hw is not scaled: sd = hw - d, d scales with s */
              dsd_ds = -(qs[a].d - (nx * rx + ny * ry)) / q[3];
            gb[4 * e + 0] += gsd * (-gx);
            gb[4 * e + 1] += gsd * (-gy);
            gb[4 * e + 2] += gsd * dsd_dth;
            gb[4 * e + 3] += gsd * dsd_ds;
          }
        }
      }
      free(list);
      free(qs);
      free(cs);
      free(cps);
      free(sds);
    }
    /* fixed-order reduction over threads */
    double* gvsum = (double*)calloc(2 * (size_t)(V > 0 ? V : 1), sizeof(double));
    for (int t = 0; t < nth; ++t)
      for (long k = 0; k < 2L * V; ++k) gvsum[k] += acc_v[(size_t)t * 2 * V + k];
    if (grad_v)
      for (long k = 0; k < 2L * V; ++k) grad_v[k] = gvsum[k];
    if (grad_b) {
      for (long k = 0; k < 4L * n; ++k) grad_b[k] = 0.0;
      for (int t = 0; t < nth; ++t)
        for (long k = 0; k < 4L * n; ++k) grad_b[k] += acc_b[(size_t)t * 4 * n + k];
    }
    if (grad_a) {
      /* Jacobian of Eq. 2: dP'/dt = I, dP'/dtheta = J r (s P), dP'/ds = r P */
      for (int e = 0; e < n; ++e) {
        const double* q = params + 4 * e;
        double c = cos(q[2]), sn = sin(q[2]), s = q[3];
        double gt0 = 0, gt1 = 0, gth = 0, gs = 0;
        for (int k = sc->voff[e]; k < sc->voff[e + 1]; ++k) {
          double gx = gvsum[2 * k], gy = gvsum[2 * k + 1];
          double rvx = c * sc->vloc[k].x - sn * sc->vloc[k].y; /* r P */
          double rvy = sn * sc->vloc[k].x + c * sc->vloc[k].y;
          gt0 += gx;
          gt1 += gy;
          gth += gx * (-s * rvy) + gy * (s * rvx);
          gs += gx * rvx + gy * rvy;
        }
        grad_a[4 * e] = gt0;
        grad_a[4 * e + 1] = gt1;
        grad_a[4 * e + 2] = gth;
        grad_a[4 * e + 3] = gs;
      }
    }
    free(gvsum);
    free(acc_v);
    free(acc_b);
    free(gI);
    free(gA);
  }
  free(gou);
  free(covc);
  free(ihat);
  free(atau);
  free(occ);
  free_world(&g);
}

/* ---------------------------------------------------------------------------------------------
 * Adam (Kingma & Ba 2015, bias-corrected), standing in for the plain descent step of Eq. 4
 * ------------------------------------------------------------------------------------------- */
void ora_adam(int n, double* p, double* m, double* v, const double* g, int step, double lr,
              double b1, double b2, double eps, const unsigned char* trainable, double s_min,
              double s_max) {
  double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
  for (int k = 0; k < 4 * n; ++k) {
    if (trainable && !trainable[k]) continue;
    m[k] = b1 * m[k] + (1.0 - b1) * g[k];
    v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
    double mh = m[k] / bc1, vh = v[k] / bc2;
    p[k] -= lr * mh / (sqrt(vh) + eps);
    if (k % 4 == 3) {
      if (p[k] < s_min) p[k] = s_min;
      if (p[k] > s_max) p[k] = s_max;
    }
  }
}

/* ---------------------------------------------------------------------------------------------
 * Binning rule (float arithmetic in this exact order; compiled without contraction):
 *   R_px = (s * r_bin) * res, cx = tx * res, cy = ty * res,
 *   m = ((rho_px + pad_px) + hw * res) + 1       (hw = 0 for closed outlines)
 *   x0 = (cx - R_px) - m, x1 = (cx + R_px) + m   (same for y)
 *   tile range [floor(x0 / T), floor(x1 / T)] clipped to the grid's tiles; empty if it misses.
 * r_bin = the largest |control point| bounds the outline (a Bezier curve stays in the convex hull
 * of its control points), so the circle of radius s r_bin about t holds the element.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  int tx0, tx1, ty0, ty1;
} tile_rect;

static tile_rect bin_rect(const ora_scene* sc, const float* params, int e, int res, int T,
                          float rho_px, float pad_px) {
  tile_rect r = {0, -1, 0, -1};
  int nt = (res + T - 1) / T;
  float fres = (float)res;
  float tx = params[4 * e], ty = params[4 * e + 1], s = params[4 * e + 3];
  float hw = is_closed(sc->kind[e]) ? 0.0f : (float)sc->hw[e];
  float Rpx = (s * sc->rbin[e]) * fres;
  float cx = tx * fres, cy = ty * fres;
  float m = ((rho_px + pad_px) + hw * fres) + 1.0f;
  float x0 = (cx - Rpx) - m, x1 = (cx + Rpx) + m;
  float y0 = (cy - Rpx) - m, y1 = (cy + Rpx) + m;
  float fT = (float)T;
  float fx0 = floorf(x0 / fT), fx1 = floorf(x1 / fT), fy0 = floorf(y0 / fT), fy1 = floorf(y1 / fT);
  float lim = (float)(nt - 1);
  if (!(fx1 >= 0.0f && fy1 >= 0.0f && fx0 <= lim && fy0 <= lim)) return r; /* also catches NaN */
  r.tx0 = fx0 < 0.0f ? 0 : (int)fx0;
  r.ty0 = fy0 < 0.0f ? 0 : (int)fy0;
  r.tx1 = fx1 > lim ? nt - 1 : (int)fx1;
  r.ty1 = fy1 > lim ? nt - 1 : (int)fy1;
  return r;
}

static int cmp_pair(const void* a, const void* b) {
  const int* x = (const int*)a;
  const int* y = (const int*)b;
  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
  if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
  return 0;
}

static long finish_pairs(int* pr, long cnt, int* tile_out, int* elem_out, long cap) {
  qsort(pr, (size_t)cnt, 2 * sizeof(int), cmp_pair);
  for (long k = 0; k < cnt && k < cap; ++k) {
    tile_out[k] = pr[2 * k];
    elem_out[k] = pr[2 * k + 1];
  }
  free(pr);
  return cnt;
}

long ora_bins(const ora_scene* sc, const float* params, int res, int T, float rho_px,
              float pad_px, int* tile_out, int* elem_out, long cap) {
  int nt = (res + T - 1) / T;
  long cnt = 0;
  for (int e = 0; e < sc->n; ++e) {
    tile_rect r = bin_rect(sc, params, e, res, T, rho_px, pad_px);
    if (r.tx1 >= r.tx0 && r.ty1 >= r.ty0) cnt += (long)(r.tx1 - r.tx0 + 1) * (r.ty1 - r.ty0 + 1);
  }
  int* pr = (int*)malloc(sizeof(int) * 2 * (cnt > 0 ? cnt : 1));
  long w = 0;
  for (int e = 0; e < sc->n; ++e) {
    tile_rect r = bin_rect(sc, params, e, res, T, rho_px, pad_px);
    for (int ty = r.ty0; ty <= r.ty1; ++ty)
      for (int tx = r.tx0; tx <= r.tx1; ++tx) {
        pr[2 * w] = ty * nt + tx;
        pr[2 * w + 1] = e;
        ++w;
      }
  }
  return finish_pairs(pr, cnt, tile_out, elem_out, cap);
}

long ora_bins_bruteforce(const ora_scene* sc, const float* params, int res, int T, float rho_px,
                         float pad_px, int* tile_out, int* elem_out, long cap) {
  int nt = (res + T - 1) / T;
  long cnt = 0, alloc = 1024;
  int* pr = (int*)malloc(sizeof(int) * 2 * alloc);
  float fres = (float)res;
  for (int e = 0; e < sc->n; ++e) {
    float tx = params[4 * e], ty = params[4 * e + 1], s = params[4 * e + 3];
    float hw = is_closed(sc->kind[e]) ? 0.0f : (float)sc->hw[e];
    float Rpx = (s * sc->rbin[e]) * fres;
    float cx = tx * fres, cy = ty * fres;
    float m = ((rho_px + pad_px) + hw * fres) + 1.0f;
    float x0 = (cx - Rpx) - m, x1 = (cx + Rpx) + m;
    float y0 = (cy - Rpx) - m, y1 = (cy + Rpx) + m;
    for (int ty_ = 0; ty_ < nt; ++ty_)
      for (int tx_ = 0; tx_ < nt; ++tx_) {
        /* tile [tx_*T, (tx_+1)*T) overlaps [x0, x1] (closed) */
        float a0 = (float)(tx_ * T), a1 = (float)((tx_ + 1) * T);
        float b0 = (float)(ty_ * T), b1 = (float)((ty_ + 1) * T);
        if (x1 >= a0 && x0 < a1 && y1 >= b0 && y0 < b1) {
          if (cnt == alloc) {
            alloc *= 2;
            pr = (int*)realloc(pr, sizeof(int) * 2 * alloc);
          }
          pr[2 * cnt] = ty_ * nt + tx_;
          pr[2 * cnt + 1] = e;
          ++cnt;
        }
      }
  }
  return finish_pairs(pr, cnt, tile_out, elem_out, cap);
}

double ora_pair_work(const ora_scene* sc, const double* params, int R, const ora_opts* o) {
  double rho = o->rho_px / R, pad = o->pad_px / R;
  world_geom g = make_world(sc, params, rho, pad);
  double work = 0.0;
  for (int e = 0; e < sc->n; ++e) {
    const double* b = g.box + 4 * e;
    /* pixel centres (j + 1/2)/R inside [b0, b2] */
    long j0 = (long)ceil(b[0] * R - 0.5), j1 = (long)floor(b[2] * R - 0.5);
    long i0 = (long)ceil(b[1] * R - 0.5), i1 = (long)floor(b[3] * R - 0.5);
    if (j0 < 0) j0 = 0;
    if (i0 < 0) i0 = 0;
    if (j1 > R - 1) j1 = R - 1;
    if (i1 > R - 1) i1 = R - 1;
    if (j1 < j0 || i1 < i0) continue;
    work += (double)(j1 - j0 + 1) * (double)(i1 - i0 + 1) * (double)n_segs(sc, e);
  }
  free_world(&g);
  return work;
}

/* ---------------------------------------------------------------------------------------------
 * Quality metrics (Sec. 6 and Sec. 6.1)
 * ------------------------------------------------------------------------------------------- */
void ora_metrics(const ora_scene* sc, const double* params, int R, const ora_opts* o, double* out,
                 unsigned char* obj_out, unsigned char* shape_out) {
  double rho = o->rho_px / R, pad = o->pad_px / R;
  long NP = (long)R * R;
  double* covc = (double*)malloc(sizeof(double) * NP);
  unsigned char* obj = (unsigned char*)malloc(NP);
  unsigned char* over = (unsigned char*)malloc(NP);
  container_images(sc, R, rho, covc);
  world_geom g = make_world(sc, params, rho, pad);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < R; ++j) {
      vec2 p = pixel_centre(i, j, R);
      double keep = 1.0;
      int n_in = 0;
      for (int e = 0; e < sc->n; ++e) {
        if (o->cull && culled(&g, e, p)) continue;
        chain_query cq = element_query(sc, e, g.wv + sc->voff[e], p);
        double sd = element_sd(sc, e, &cq);
        keep *= 1.0 - S(sd / rho);
        if (sd >= 0.0) n_in += 1;
      }
      obj[(long)i * R + j] = 1.0 - keep >= 0.5;
      over[(long)i * R + j] = n_in >= 2;
    }
  free_world(&g);
  double n_obj_in = 0, n_shape = 0, n_over = 0, n_exceed = 0;
  for (long p = 0; p < NP; ++p) {
    int shape = covc[p] >= 0.5;
    n_shape += shape;
    n_obj_in += shape && obj[p];
    n_exceed += !shape && obj[p];
    n_over += over[p];
  }
  out[0] = n_obj_in;
  out[1] = n_shape;
  out[2] = n_over;
  out[3] = n_exceed;
  out[4] = n_shape > 0 ? n_obj_in / n_shape : 0.0;
  out[5] = n_shape > 0 ? n_over / n_shape : 0.0;
  out[6] = n_shape > 0 ? n_exceed / n_shape : 0.0;
  out[7] = 0.0;
  for (long p = 0; p < NP; ++p) {
    if (obj_out) obj_out[p] = obj[p];
    if (shape_out) shape_out[p] = covc[p] >= 0.5;
  }
  free(covc);
  free(obj);
  free(over);
}

int ora_set_threads(int n) {
  const int prev = omp_get_max_threads();
  omp_set_num_threads(n >= 1 ? n : omp_get_num_procs());
  return prev;
}
