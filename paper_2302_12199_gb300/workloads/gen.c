/*
 * Seeded synthetic graph generators: GNM, 2D/3D random geometric (RGG), RMAT,
 * 2D grids, random hyperbolic graphs (RHG) and the mixed batches of many small
 * graphs.
 *
 * These stand in for the graph families of the paper's experiments (Section 7,
 * "Instances and Methodology": KaGen GNM / RGG generators and an RMAT generator
 * with the Graph500 probabilities, weights uniform in [1,255)).  The paper's
 * real-world graphs are not used.
 *
 * This module holds input generation only: no step of any MST method.  Both the
 * CPU oracle tests and the GPU path take their inputs from here.
 *
 * Randomness is counter based: output i of the splitmix64 sequence started at
 * state s is mix(s + (i+1) * 0x9e3779b97f4a7c15), where mix is splitmix64's
 * finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014).  Every draw is addressed by (stream, index), so the
 * output does not depend on the thread count.  Floating point is only used for
 * RGG coordinates and distances; the file is compiled with -ffp-contract=off so
 * that x86-64 and aarch64 produce identical graphs.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9e3779b97f4a7c15ULL

static inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* output #i of the splitmix64 sequence whose state starts at s */
static inline uint64_t sm_at(uint64_t s, uint64_t i) { return sm_mix(s + (i + 1) * GOLDEN); }

/* independent sub-stream state for a (seed, tag) pair */
static inline uint64_t sub_seed(uint64_t seed, uint64_t tag) { return sm_mix(seed ^ sm_mix(tag + GOLDEN)); }

/* uniform integer in [0, r) by multiply-shift (Lemire) */
static inline uint64_t bounded(uint64_t x, uint64_t r) {
  return (uint64_t)(((unsigned __int128)x * (unsigned __int128)r) >> 64);
}

uint64_t gen_splitmix64_at(uint64_t s, uint64_t i) { return sm_at(s, i); }

/* Stream tags. */
enum { TAG_U = 1, TAG_V = 2, TAG_W = 3, TAG_PERM = 4, TAG_X = 5, TAG_Y = 6, TAG_Z = 7, TAG_GRAPH = 8, TAG_EDGE = 9 };

/* ------------------------------------------------------------------ threads */

typedef struct {
  void (*fn)(void *ctx, uint64_t lo, uint64_t hi);
  void *ctx;
  uint64_t lo, hi;
} job_t;

static void *job_run(void *p) {
  job_t *j = (job_t *)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void parallel_for(uint64_t count, int nthreads, void (*fn)(void *, uint64_t, uint64_t), void *ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  if (count < (uint64_t)nthreads * 65536ULL) nthreads = 1;
  if (nthreads == 1) {
    fn(ctx, 0, count);
    return;
  }
  pthread_t th[64];
  job_t jobs[64];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].lo = count * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].hi = count * (uint64_t)(t + 1) / (uint64_t)nthreads;
    pthread_create(&th[t], NULL, job_run, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ---------------------------------------------------------------------- GNM */

typedef struct {
  uint64_t n, wmin, wspan, su, sw;
  uint32_t *src, *dst, *w;
} gnm_ctx;

static void gnm_body(void *p, uint64_t lo, uint64_t hi) {
  gnm_ctx *c = (gnm_ctx *)p;
  for (uint64_t i = lo; i < hi; ++i) {
    uint64_t es = sub_seed(c->su, i);
    uint64_t u = bounded(sm_at(es, 0), c->n);
    uint64_t v = bounded(sm_at(es, 1), c->n);
    /* self-loops are redrawn (a bounded number of times) so that m stays exact */
    for (uint64_t k = 2; u == v && c->n > 1 && k < 256; ++k) v = bounded(sm_at(es, k), c->n);
    c->src[i] = (uint32_t)u;
    c->dst[i] = (uint32_t)v;
    c->w[i] = (uint32_t)(c->wmin + bounded(sm_at(c->sw, i), c->wspan));
  }
}

/* G(n,m): m endpoint pairs drawn uniformly, duplicates kept, self-loops redrawn;
 * weights uniform in [wmin, wmax]. */
void gen_gnm(uint64_t n, uint64_t m, uint64_t seed, uint32_t wmin, uint32_t wmax, int nthreads, uint32_t *src,
             uint32_t *dst, uint32_t *w) {
  gnm_ctx c = {n, wmin, (uint64_t)wmax - wmin + 1, sub_seed(seed, TAG_U), sub_seed(seed, TAG_W), src, dst, w};
  parallel_for(m, nthreads, gnm_body, &c);
}

/* --------------------------------------------------------------------- RMAT */

typedef struct {
  int scale;
  uint64_t n, wmin, wspan, se, sw;
  uint32_t ta, tb, tc;
  const uint32_t *perm;
  uint32_t *src, *dst, *w;
} rmat_ctx;

static void rmat_body(void *p, uint64_t lo, uint64_t hi) {
  rmat_ctx *c = (rmat_ctx *)p;
  for (uint64_t i = lo; i < hi; ++i) {
    uint64_t es = sub_seed(c->se, i);
    uint64_t u = 0, v = 0, bits = 0;
    for (int l = 0; l < c->scale; ++l) {
      if ((l & 3) == 0) bits = sm_at(es, (uint64_t)(l >> 2));
      uint32_t t = (uint32_t)(bits & 0xffff);
      bits >>= 16;
      uint64_t bu = 0, bv = 0;
      if (t < c->ta) {
      } else if (t < c->tb) {
        bv = 1;
      } else if (t < c->tc) {
        bu = 1;
      } else {
        bu = 1;
        bv = 1;
      }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    if (u >= c->n) u %= c->n; /* fold when n is not a power of two */
    if (v >= c->n) v %= c->n;
    c->src[i] = c->perm ? c->perm[u] : (uint32_t)u;
    c->dst[i] = c->perm ? c->perm[v] : (uint32_t)v;
    c->w[i] = (uint32_t)(c->wmin + bounded(sm_at(c->sw, i), c->wspan));
  }
}

static uint32_t prob16(double p) {
  double t = p * 65536.0 + 0.5;
  if (t < 0) t = 0;
  if (t > 65536.0) t = 65536.0;
  return (uint32_t)t;
}

/* RMAT: each of the `scale` levels picks a quadrant of the adjacency matrix with
 * probabilities (a,b,c,1-a-b-c), quantised to 1/65536.  Vertex ids are then
 * mapped through a seeded random permutation of 0..n-1 when `permute` is set.
 * Self-loops and duplicates are kept as drawn. */
void gen_rmat(int scale, uint64_t n, uint64_t m, double a, double b, double c, int permute, uint64_t seed,
              uint32_t wmin, uint32_t wmax, int nthreads, uint32_t *src, uint32_t *dst, uint32_t *w) {
  uint32_t *perm = NULL;
  if (permute) {
    perm = (uint32_t *)malloc(n * sizeof(uint32_t));
    for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    uint64_t sp = sub_seed(seed, TAG_PERM);
    for (uint64_t i = n; i > 1; --i) { /* Fisher-Yates */
      uint64_t j = bounded(sm_at(sp, i - 1), i);
      uint32_t t = perm[i - 1];
      perm[i - 1] = perm[j];
      perm[j] = t;
    }
  }
  rmat_ctx x;
  x.scale = scale;
  x.n = n;
  x.wmin = wmin;
  x.wspan = (uint64_t)wmax - wmin + 1;
  x.se = sub_seed(seed, TAG_EDGE);
  x.sw = sub_seed(seed, TAG_W);
  x.ta = prob16(a);
  x.tb = prob16(a + b);
  x.tc = prob16(a + b + c);
  x.perm = perm;
  x.src = src;
  x.dst = dst;
  x.w = w;
  parallel_for(m, nthreads, rmat_body, &x);
  free(perm);
}

/* ---------------------------------------------------------------------- RGG */

/* Points uniform in [0,1)^dim with f32 coordinates (24 random mantissa bits).
 * Vertices are numbered cell by cell (cells of side >= r), the cells taken in
 * Morton (Z) order, so that a range of consecutive ids covers a compact square
 * (cube) of the domain, like the spatial partition KaGen gives each PE.  Every
 * pair at Euclidean distance < r becomes one undirected edge (u < v), emitted
 * in ascending u.  Returns the number of edges; with src == NULL only counts. */
static float coord(uint64_t s, uint64_t i) { return (float)((double)(sm_at(s, i) >> 40) * (1.0 / 16777216.0)); }

typedef struct {
  int dim;
  uint64_t n, G, ncell;
  double r2;
  float *x, *y, *z;      /* by new id */
  uint64_t *cell_start;  /* [ncell] first new id of each (row-major) cell */
  uint64_t *cell_end;    /* [ncell] one past its last */
} rgg_t;

static uint64_t cell_of(const rgg_t *g, double x, double y, double z) {
  uint64_t cx = (uint64_t)(x * (double)g->G), cy = (uint64_t)(y * (double)g->G), cz = 0;
  if (cx >= g->G) cx = g->G - 1;
  if (cy >= g->G) cy = g->G - 1;
  if (g->dim == 3) {
    cz = (uint64_t)(z * (double)g->G);
    if (cz >= g->G) cz = g->G - 1;
  }
  return (cz * g->G + cy) * g->G + cx;
}

/* Morton code: bit b of coordinate k goes to bit b*dim + k. */
static uint64_t morton(uint64_t cx, uint64_t cy, uint64_t cz, int dim) {
  uint64_t code = 0;
  for (int b = 0; b < 21; ++b) {
    code |= ((cx >> b) & 1ULL) << (b * dim);
    code |= ((cy >> b) & 1ULL) << (b * dim + 1);
    if (dim == 3) code |= ((cz >> b) & 1ULL) << (b * dim + 2);
  }
  return code;
}

typedef struct {
  uint64_t code, cell;
} cell_key_t;

static int cmp_cell_key(const void *a, const void *b) {
  const cell_key_t *x = (const cell_key_t *)a, *y = (const cell_key_t *)b;
  return x->code < y->code ? -1 : (x->code > y->code ? 1 : 0);
}

static int rgg_build(rgg_t *g, int dim, uint64_t n, double r, uint64_t seed) {
  g->dim = dim;
  g->n = n;
  g->r2 = r * r;
  uint64_t G = (uint64_t)floor(1.0 / r);
  if (G < 1) G = 1;
  if (dim == 2 && G > 8192) G = 8192;
  if (dim == 3 && G > 512) G = 512;
  g->G = G;
  g->ncell = dim == 2 ? G * G : G * G * G;
  uint64_t sx = sub_seed(seed, TAG_X), sy = sub_seed(seed, TAG_Y), sz = sub_seed(seed, TAG_Z);
  float *x0 = (float *)malloc(n * sizeof(float)), *y0 = (float *)malloc(n * sizeof(float));
  float *z0 = dim == 3 ? (float *)malloc(n * sizeof(float)) : NULL;
  uint64_t *cell = (uint64_t *)malloc(n * sizeof(uint64_t));
  uint64_t *cnt = (uint64_t *)calloc(g->ncell, sizeof(uint64_t));
  g->cell_start = (uint64_t *)malloc(g->ncell * sizeof(uint64_t));
  g->cell_end = (uint64_t *)malloc(g->ncell * sizeof(uint64_t));
  g->x = (float *)malloc(n * sizeof(float));
  g->y = (float *)malloc(n * sizeof(float));
  g->z = dim == 3 ? (float *)malloc(n * sizeof(float)) : NULL;
  for (uint64_t i = 0; i < n; ++i) {
    x0[i] = coord(sx, i);
    y0[i] = coord(sy, i);
    if (dim == 3) z0[i] = coord(sz, i);
    cell[i] = cell_of(g, x0[i], y0[i], dim == 3 ? z0[i] : 0.0);
    cnt[cell[i]]++;
  }
  /* cells in Morton order; each cell's points get a contiguous id range */
  cell_key_t *keys = (cell_key_t *)malloc(g->ncell * sizeof(cell_key_t));
  for (uint64_t c = 0; c < g->ncell; ++c) {
    keys[c].code = morton(c % G, (c / G) % G, c / (G * G), dim);
    keys[c].cell = c;
  }
  qsort(keys, g->ncell, sizeof(cell_key_t), cmp_cell_key);
  uint64_t next = 0;
  for (uint64_t k = 0; k < g->ncell; ++k) {
    const uint64_t c = keys[k].cell;
    g->cell_start[c] = next;
    next += cnt[c];
    g->cell_end[c] = next;
  }
  free(keys);
  uint64_t *fill = (uint64_t *)malloc(g->ncell * sizeof(uint64_t));
  memcpy(fill, g->cell_start, g->ncell * sizeof(uint64_t));
  for (uint64_t i = 0; i < n; ++i) { /* stable within each cell */
    uint64_t id = fill[cell[i]]++;
    g->x[id] = x0[i];
    g->y[id] = y0[i];
    if (dim == 3) g->z[id] = z0[i];
  }
  free(fill);
  free(cnt);
  free(cell);
  free(x0);
  free(y0);
  free(z0);
  return 0;
}

static void rgg_free(rgg_t *g) {
  free(g->x);
  free(g->y);
  free(g->z);
  free(g->cell_start);
  free(g->cell_end);
}

static uint64_t rgg_edges(const rgg_t *g, uint32_t *src, uint32_t *dst) {
  uint64_t cnt = 0, G = g->G;
  for (uint64_t p = 0; p < g->n; ++p) {
    double px = g->x[p], py = g->y[p], pz = g->dim == 3 ? g->z[p] : 0.0;
    uint64_t c = cell_of(g, px, py, pz);
    int64_t cx = (int64_t)(c % G), cy = (int64_t)((c / G) % G), cz = (int64_t)(c / (G * G));
    int zlo = g->dim == 3 ? -1 : 0, zhi = g->dim == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int64_t nx = cx + dx, ny = cy + dy, nz = cz + dz;
          if (nx < 0 || ny < 0 || nz < 0 || nx >= (int64_t)G || ny >= (int64_t)G || nz >= (int64_t)G) continue;
          uint64_t nc = ((uint64_t)nz * G + (uint64_t)ny) * G + (uint64_t)nx;
          for (uint64_t q = g->cell_start[nc]; q < g->cell_end[nc]; ++q) {
            if (q <= p) continue;
            double ddx = px - (double)g->x[q], ddy = py - (double)g->y[q];
            double d2 = ddx * ddx + ddy * ddy;
            if (g->dim == 3) {
              double ddz = pz - (double)g->z[q];
              d2 += ddz * ddz;
            }
            if (d2 < g->r2) {
              if (src) {
                src[cnt] = (uint32_t)p;
                dst[cnt] = (uint32_t)q;
              }
              ++cnt;
            }
          }
        }
  }
  return cnt;
}

/* Count pass: number of edges of the RGG (dim 2 or 3). */
uint64_t gen_rgg_count(int dim, uint64_t n, double r, uint64_t seed) {
  rgg_t g;
  rgg_build(&g, dim, n, r, seed);
  uint64_t c = rgg_edges(&g, NULL, NULL);
  rgg_free(&g);
  return c;
}

/* Fill pass: writes exactly gen_rgg_count(...) edges; weights uniform in [wmin,wmax]. */
uint64_t gen_rgg_fill(int dim, uint64_t n, double r, uint64_t seed, uint32_t wmin, uint32_t wmax, uint32_t *src,
                      uint32_t *dst, uint32_t *w) {
  rgg_t g;
  rgg_build(&g, dim, n, r, seed);
  uint64_t c = rgg_edges(&g, src, dst);
  rgg_free(&g);
  uint64_t sw = sub_seed(seed, TAG_W), span = (uint64_t)wmax - wmin + 1;
  for (uint64_t i = 0; i < c; ++i) w[i] = (uint32_t)(wmin + bounded(sm_at(sw, i), span));
  return c;
}

/* ------------------------------------------------------------------ 2D grid */

/* rows x cols grid, vertex r*cols + c; edges to the right and lower neighbour
 * (in that order per vertex), rows*(cols-1) + (rows-1)*cols in all; weights
 * uniform in [wmin, wmax].  Standing in for the paper's 2D-grid family. */
uint64_t gen_grid2d(uint64_t rows, uint64_t cols, uint64_t seed, uint32_t wmin, uint32_t wmax, uint32_t *src,
                    uint32_t *dst, uint32_t *w) {
  const uint64_t m = rows * (cols ? cols - 1 : 0) + (rows ? rows - 1 : 0) * cols;
  if (!src) return m;
  const uint64_t sw = sub_seed(seed, TAG_W), span = (uint64_t)wmax - wmin + 1;
  uint64_t k = 0;
  for (uint64_t r = 0; r < rows; ++r)
    for (uint64_t c = 0; c < cols; ++c) {
      const uint64_t v = r * cols + c;
      if (c + 1 < cols) {
        src[k] = (uint32_t)v;
        dst[k] = (uint32_t)(v + 1);
        w[k] = (uint32_t)(wmin + bounded(sm_at(sw, k), span));
        ++k;
      }
      if (r + 1 < rows) {
        src[k] = (uint32_t)v;
        dst[k] = (uint32_t)(v + cols);
        w[k] = (uint32_t)(wmin + bounded(sm_at(sw, k), span));
        ++k;
      }
    }
  return k;
}

/* ------------------------------------------------- random hyperbolic graph */

/* Threshold random hyperbolic graph in the hyperbolic plane (curvature -1):
 * n points in a disk of radius R, angle uniform, radius with density
 * alpha sinh(alpha r) / (cosh(alpha R) - 1) (power-law degrees with exponent
 * gamma = 2 alpha + 1), an edge between two points closer than R.  Vertices are
 * numbered in angular order.  Standing in for the paper's RHG family.  Uses
 * libm (cosh, sinh, acosh, cos): graphs are identical on hosts with the same
 * libm.  Neighbour search: radial bands of width 1; for a query point, a band
 * is scanned over the angular window its inner radius allows. */
typedef struct {
  uint64_t n;
  double R, coshR;
  double *theta, *chr, *shr; /* per vertex (angular order) */
  int nb;                    /* bands */
  double *b_lo;              /* inner radius of each band */
  uint64_t *b_start;         /* band members: positions b_start[j] .. b_start[j+1]-1 in b_idx */
  uint32_t *b_idx;           /* vertex ids, ascending angle within a band */
  double *b_theta;
} rhg_t;

typedef struct {
  double th;
  double r;
} pt_t;

static int cmp_pt(const void *a, const void *b) {
  const pt_t *x = (const pt_t *)a, *y = (const pt_t *)b;
  return x->th < y->th ? -1 : x->th > y->th ? 1 : 0;
}

static void rhg_build(rhg_t *g, uint64_t n, double alpha, double R, uint64_t seed) {
  const double two_pi = 6.283185307179586476925286766559;
  g->n = n;
  g->R = R;
  g->coshR = cosh(R);
  pt_t *pts = (pt_t *)malloc(sizeof(pt_t) * (n ? n : 1));
  const uint64_t s1 = sub_seed(seed, TAG_X), s2 = sub_seed(seed, TAG_Y);
  const double cmax = cosh(alpha * R) - 1.0;
  for (uint64_t i = 0; i < n; ++i) {
    const double u1 = (double)(sm_at(s1, i) >> 11) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(sm_at(s2, i) >> 11) * (1.0 / 9007199254740992.0);
    pts[i].th = two_pi * u1;
    pts[i].r = acosh(1.0 + u2 * cmax) / alpha;
  }
  qsort(pts, n, sizeof(pt_t), cmp_pt);
  g->theta = (double *)malloc(sizeof(double) * (n ? n : 1));
  g->chr = (double *)malloc(sizeof(double) * (n ? n : 1));
  g->shr = (double *)malloc(sizeof(double) * (n ? n : 1));
  for (uint64_t i = 0; i < n; ++i) {
    g->theta[i] = pts[i].th;
    g->chr[i] = cosh(pts[i].r);
    g->shr[i] = sinh(pts[i].r);
  }
  /* bands [R-1, R], [R-2, R-1], ..., [0, ...] */
  g->nb = (int)ceil(R);
  if (g->nb < 1) g->nb = 1;
  g->b_lo = (double *)malloc(sizeof(double) * g->nb);
  for (int j = 0; j < g->nb; ++j) {
    const double lo = R - (double)(j + 1);
    g->b_lo[j] = lo > 0.0 ? lo : 0.0;
  }
  g->b_start = (uint64_t *)calloc(g->nb + 1, sizeof(uint64_t));
  int *band = (int *)malloc(sizeof(int) * (n ? n : 1));
  for (uint64_t i = 0; i < n; ++i) {
    int j = (int)(R - pts[i].r);
    if (j < 0) j = 0;
    if (j >= g->nb) j = g->nb - 1;
    band[i] = j;
    g->b_start[j + 1]++;
  }
  for (int j = 0; j < g->nb; ++j) g->b_start[j + 1] += g->b_start[j];
  uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * g->nb);
  for (int j = 0; j < g->nb; ++j) fill[j] = g->b_start[j];
  g->b_idx = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  g->b_theta = (double *)malloc(sizeof(double) * (n ? n : 1));
  for (uint64_t i = 0; i < n; ++i) { /* ascending angle within each band (vertex order is angular) */
    const uint64_t at = fill[band[i]]++;
    g->b_idx[at] = (uint32_t)i;
    g->b_theta[at] = g->theta[i];
  }
  free(fill);
  free(band);
  free(pts);
}

static void rhg_free(rhg_t *g) {
  free(g->theta);
  free(g->chr);
  free(g->shr);
  free(g->b_lo);
  free(g->b_start);
  free(g->b_idx);
  free(g->b_theta);
}

static uint64_t lower_theta(const double *a, uint64_t lo, uint64_t hi, double x) {
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (a[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

/* Neighbours q > p of vertex p (each undirected edge once), in band order and
 * ascending angle within a band; writes them to out (if non-null); returns the count. */
static uint64_t rhg_neighbours(const rhg_t *g, uint64_t p, uint32_t *out) {
  const double pi = 3.141592653589793238462643383279, two_pi = 2.0 * pi;
  const double tp = g->theta[p], chp = g->chr[p], shp = g->shr[p];
  uint64_t c = 0;
  for (int j = 0; j < g->nb; ++j) {
    const uint64_t lo = g->b_start[j], hi = g->b_start[j + 1];
    if (lo == hi) continue;
    /* widest angle at which a point of radius >= b_lo[j] can still be closer than R */
    const double rl = g->b_lo[j];
    double width = pi;
    const double sh = shp * sinh(rl);
    if (sh > 0.0) {
      const double cth = (chp * cosh(rl) - g->coshR) / sh;
      if (cth >= 1.0) continue;
      if (cth > -1.0) width = acos(cth);
    }
    /* the window [tp - width, tp + width] on the circle, as at most two ranges */
    double a0 = tp - width, a1 = tp + width;
    double ranges[2][2];
    int nr = 0;
    if (width >= pi) {
      ranges[nr][0] = 0.0;
      ranges[nr][1] = two_pi;
      ++nr;
    } else if (a0 < 0.0) {
      ranges[nr][0] = 0.0, ranges[nr][1] = a1, ++nr;
      ranges[nr][0] = a0 + two_pi, ranges[nr][1] = two_pi, ++nr;
    } else if (a1 > two_pi) {
      ranges[nr][0] = a0, ranges[nr][1] = two_pi, ++nr;
      ranges[nr][0] = 0.0, ranges[nr][1] = a1 - two_pi, ++nr;
    } else {
      ranges[nr][0] = a0, ranges[nr][1] = a1, ++nr;
    }
    for (int k = 0; k < nr; ++k) {
      uint64_t at = lower_theta(g->b_theta, lo, hi, ranges[k][0]);
      for (; at < hi && g->b_theta[at] <= ranges[k][1]; ++at) {
        const uint64_t q = g->b_idx[at];
        if (q <= p) continue;
        const double dth = fabs(g->theta[q] - tp);
        const double cd = chp * g->chr[q] - shp * g->shr[q] * cos(dth);
        if (cd < g->coshR) {
          if (out) out[c] = (uint32_t)q;
          ++c;
        }
      }
    }
  }
  return c;
}

typedef struct {
  const rhg_t *g;
  uint64_t *count; /* per vertex */
  const uint64_t *off;
  uint32_t *src, *dst;
} rhg_job_t;

static void rhg_count_body(void *p, uint64_t lo, uint64_t hi) {
  rhg_job_t *j = (rhg_job_t *)p;
  for (uint64_t v = lo; v < hi; ++v) j->count[v] = rhg_neighbours(j->g, v, NULL);
}

static void rhg_fill_body(void *p, uint64_t lo, uint64_t hi) {
  rhg_job_t *j = (rhg_job_t *)p;
  for (uint64_t v = lo; v < hi; ++v) {
    const uint64_t o = j->off[v];
    const uint64_t c = rhg_neighbours(j->g, v, j->dst + o);
    for (uint64_t k = 0; k < c; ++k) j->src[o + k] = (uint32_t)v;
  }
}

/* Radius giving expected average degree deg for alpha (Krioukov et al. 2010,
 * the large-n form k = xi^2 (2/pi) n e^{-R/2}, xi = alpha / (alpha - 1/2)). */
double gen_rhg_radius(uint64_t n, double deg, double alpha) {
  const double pi = 3.141592653589793238462643383279;
  const double xi = alpha / (alpha - 0.5);
  return 2.0 * log(xi * xi * 2.0 / pi * (double)n / deg);
}

/* Two passes as for RGG: with src == NULL returns the edge count only. */
uint64_t gen_rhg(uint64_t n, double alpha, double R, uint64_t seed, uint32_t wmin, uint32_t wmax, int nthreads,
                 uint32_t *src, uint32_t *dst, uint32_t *w) {
  rhg_t g;
  rhg_build(&g, n, alpha, R, seed);
  uint64_t *count = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
  rhg_job_t job = {&g, count, NULL, NULL, NULL};
  parallel_for(n, nthreads, rhg_count_body, &job);
  uint64_t *off = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
  off[0] = 0;
  for (uint64_t v = 0; v < n; ++v) off[v + 1] = off[v] + count[v];
  const uint64_t m = off[n];
  if (src) {
    job.off = off;
    job.src = src;
    job.dst = dst;
    parallel_for(n, nthreads, rhg_fill_body, &job);
    const uint64_t sw = sub_seed(seed, TAG_W), span = (uint64_t)wmax - wmin + 1;
    for (uint64_t i = 0; i < m; ++i) w[i] = (uint32_t)(wmin + bounded(sm_at(sw, i), span));
  }
  free(off);
  free(count);
  rhg_free(&g);
  return m;
}

/* ------------------------------------------------------------ mixed batches */

/* 2^f for f in [0,1) by its Taylor series in f*ln2, evaluated with plain IEEE
 * double operations (no libm), so that the result is identical on every host. */
static double exp2_frac(double f) {
  const double ln2 = 0.69314718055994530942;
  double x = f * ln2, term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    term = term * x / (double)k;
    sum += term;
  }
  return sum;
}

typedef struct {
  uint32_t kind; /* 0 GNM, 1 RGG2D, 2 RMAT */
  uint64_t n, m, seed;
  double r;
} graph_spec_t;

static graph_spec_t mix_spec(uint64_t seed, uint64_t g, int log_lo, int log_hi) {
  graph_spec_t s;
  uint64_t gs = sub_seed(seed, (uint64_t)TAG_GRAPH * 0x100000000ULL + g);
  double t = (double)(sm_at(gs, 0) >> 11) * (1.0 / 9007199254740992.0); /* [0,1) */
  double U = (double)log_lo + (double)(log_hi - log_lo) * t;
  double ip = floor(U);
  double nv = floor(ldexp(exp2_frac(U - ip), (int)ip));
  if (nv < 2) nv = 2;
  s.n = (uint64_t)nv;
  s.kind = (uint32_t)(g % 3);
  s.seed = sm_at(gs, 1);
  s.r = 0;
  if (s.kind == 0) { /* GNM, average degree 2m/n uniform in [4,32] */
    double d = 4.0 + 28.0 * (double)(sm_at(gs, 2) >> 11) * (1.0 / 9007199254740992.0);
    s.m = (uint64_t)floor((double)s.n * d / 2.0 + 0.5);
  } else if (s.kind == 1) { /* RGG2D, expected degree 8 */
    s.r = sqrt(8.0 / (3.14159265358979323846 * (double)s.n));
    s.m = 0; /* known after the count pass */
  } else { /* RMAT, average degree 16 */
    s.m = 8 * s.n;
  }
  return s;
}

/* First pass over a mixed batch: per-graph n and m (m computed by a count pass
 * for the geometric graphs). */
void gen_mix_sizes(uint64_t seed, uint64_t num_graphs, int log_lo, int log_hi, uint32_t *n_out, uint64_t *m_out,
                   uint32_t *kind_out) {
  for (uint64_t g = 0; g < num_graphs; ++g) {
    graph_spec_t s = mix_spec(seed, g, log_lo, log_hi);
    if (s.kind == 1) s.m = gen_rgg_count(2, s.n, s.r, s.seed);
    n_out[g] = (uint32_t)s.n;
    m_out[g] = s.m;
    kind_out[g] = s.kind;
  }
}

/* Second pass: fills graph g's edges (graph-local vertex ids) at the given
 * pointers, which must hold m_out[g] entries. Weights uniform in [1,255]. */
void gen_mix_graph(uint64_t seed, uint64_t g, int log_lo, int log_hi, int nthreads, uint32_t *src, uint32_t *dst,
                   uint32_t *w) {
  graph_spec_t s = mix_spec(seed, g, log_lo, log_hi);
  if (s.kind == 0) {
    gen_gnm(s.n, s.m, s.seed, 1, 255, nthreads, src, dst, w);
  } else if (s.kind == 1) {
    gen_rgg_fill(2, s.n, s.r, s.seed, 1, 255, src, dst, w);
  } else {
    int scale = 0;
    while ((1ULL << scale) < s.n) ++scale;
    gen_rmat(scale, s.n, s.m, 0.57, 0.19, 0.19, 1, s.seed, 1, 255, nthreads, src, dst, w);
  }
}
