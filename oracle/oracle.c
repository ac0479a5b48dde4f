/*
 * Exact CPU oracle for the intersection join of closed triangle meshes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * library and it never reads a value that the CUDA path produced.
 *
 * What it computes (paper: "Pierce: GPU Ray Tracing for Spatial Joins over
 * Complex 3D Data"):
 *
 *   intersects(A,B) = cross(A,B) OR inside(B,A) OR inside(A,B)        (Sec. 3.4)
 *
 *   cross(A,B)  : some edge of A pierces a triangle of B, or some edge of B
 *                 pierces a triangle of A (Sec. 3.1 observation 1, Alg. 1
 *                 run in both directions as in Sec. 3.2 "Bidirectional
 *                 tracing").  "Pierce" is read strictly: the open segment
 *                 crosses the open triangle transversally, so tangential
 *                 contact never counts (Sec. 3.2, Sec. 3.6 "Robustness").
 *   inside(B,A) : a representative vertex of B lies inside A by the parity of
 *                 the number of triangles of A hit by a ray cast in +z
 *                 (Alg. 2, Sec. 3.3).  The parity test is not filtered by
 *                 the crossing result (Sec. 3.4).
 *
 * orc_join_pred also evaluates the paper's other two join predicates:
 * overlap = cross(A,B) (Sec. 3.2), and containment (Sec. 3.3, Alg. 2):
 * A contains B iff there is no crossing and inside(B,A); "within" is the
 * role swap.
 *
 * Coordinates are integers in [0, 2^18) (stored as float32 by callers), so
 * every orientation determinant is evaluated exactly in 64-bit integers:
 * differences are below 2^18 in magnitude, 2x2 minors below 2^37, a 3x3
 * determinant below 3 * 2^55 < 2^57.  The point-in-closed-triangle test
 * multiplies two 2^37-sized cross products and uses __int128.
 *
 * Readings of the paper (the paper works in FP32 and leaves ties to its
 * ray tracer; these are the exact rules this oracle fixes):
 *   - strict segment/triangle crossing (five orientation signs);
 *   - representative vertex = lexicographically smallest (x,y,z) vertex of B
 *     that does not lie on the closed surface of A; none -> inside = false;
 *   - the +z parity ray is perturbed symbolically to (x+e, y+e^2), so a ray
 *     through an edge or a vertex of A is counted exactly once; triangles
 *     whose xy projection has zero area never count;
 *   - zero-area triangles never produce a crossing.
 *
 * Two evaluation tiers, both single-threaded and unoptimised:
 *   tier 1: every edge (all three edges of every triangle) against every
 *           triangle, both directions, stopping at the first crossing;
 *   tier 2: the same tests restricted to edges and triangles whose closed
 *           bounding boxes meet the closed intersection of the two meshes'
 *           bounding boxes, and each other.  A strict crossing point lies in
 *           the segment, the triangle and both meshes, hence in all of those
 *           boxes, so the restriction cannot drop a crossing.
 * inside() is evaluated the same way in both tiers (all triangles).
 *
 * Every exported function is reentrant: a call reads its inputs, allocates its
 * own meshes and writes only its own outputs, so disjoint candidate lists may
 * be refined by several threads at once (the Python driver shards that way).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define ORC_GRID (1 << 18)

enum {
  ORC_OK = 0,
  ORC_ERR_RANGE = -11,    /* coordinate not an integer in [0, 2^18) */
  ORC_ERR_INDEX = -12,    /* triangle vertex index out of range      */
  ORC_ERR_ARG = -13,
  ORC_ERR_NOMEM = -14
};

typedef struct {
  const float *xyz;      /* V x 3 float32, integer valued            */
  const int32_t *tris;   /* F x 3 mesh-local vertex indices          */
  const int64_t *voff;   /* M + 1 vertex offsets                     */
  const int64_t *toff;   /* M + 1 triangle offsets                   */
  int64_t nmesh;
} orc_dataset;

/* One mesh converted to exact integer coordinates. */
typedef struct {
  int64_t nv, nf;
  int64_t *v;            /* nv x 3 */
  int32_t *t;            /* nf x 3 (local indices) */
  int64_t lo[3], hi[3];  /* closed bounding box */
} mesh_t;

static int sgn(int64_t x) { return (x > 0) - (x < 0); }

/* ---------------------------------------------------------------------- */
/* Exact primitives                                                        */
/* ---------------------------------------------------------------------- */

/* orient3d(a,b,c,d) = det [ b-a ; c-a ; d-a ] (rows).  Equals (d-a).n with
 * n = (b-a) x (c-a).  Exact: see the bound in the file header. */
int64_t orc_orient3d(const int64_t *a, const int64_t *b, const int64_t *c,
                     const int64_t *d) {
  int64_t bx = b[0] - a[0], by = b[1] - a[1], bz = b[2] - a[2];
  int64_t cx = c[0] - a[0], cy = c[1] - a[1], cz = c[2] - a[2];
  int64_t dx = d[0] - a[0], dy = d[1] - a[1], dz = d[2] - a[2];
  return bx * (cy * dz - cz * dy) - by * (cx * dz - cz * dx) +
         bz * (cx * dy - cy * dx);
}

/* orient2d in the xy plane: (b-a) x (c-a), z component. */
int64_t orc_orient2d_xy(const int64_t *a, const int64_t *b, const int64_t *c) {
  return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
}

/* Strict crossing of the open segment pq with the open triangle abc:
 * p and q strictly on opposite sides of the triangle's plane, and the line pq
 * passing strictly inside the triangle (u, v, w all nonzero, one sign). */
int32_t orc_segtri_strict(const int64_t *p, const int64_t *q, const int64_t *a,
                          const int64_t *b, const int64_t *c) {
  int sp = sgn(orc_orient3d(a, b, c, p));
  int sq = sgn(orc_orient3d(a, b, c, q));
  if (sp == 0 || sq == 0 || sp == sq) return 0;
  int u = sgn(orc_orient3d(p, q, a, b));
  int v = sgn(orc_orient3d(p, q, b, c));
  int w = sgn(orc_orient3d(p, q, c, a));
  return (u != 0 && u == v && v == w) ? 1 : 0;
}

static void cross3(const int64_t *x, const int64_t *y, int64_t *out) {
  out[0] = x[1] * y[2] - x[2] * y[1];
  out[1] = x[2] * y[0] - x[0] * y[2];
  out[2] = x[0] * y[1] - x[1] * y[0];
}
static void sub3(const int64_t *x, const int64_t *y, int64_t *out) {
  out[0] = x[0] - y[0]; out[1] = x[1] - y[1]; out[2] = x[2] - y[2];
}
static int64_t dot3(const int64_t *x, const int64_t *y) {
  return x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
}
static i128 dot3_128(const int64_t *x, const int64_t *y) {
  return (i128)x[0] * y[0] + (i128)x[1] * y[1] + (i128)x[2] * y[2];
}

/* Is v on the closed segment [s0, s1]? (s0 may equal s1.) */
static int on_closed_segment(const int64_t *v, const int64_t *s0,
                             const int64_t *s1) {
  int64_t d[3], w[3], c[3];
  sub3(s1, s0, d);
  sub3(v, s0, w);
  cross3(w, d, c);
  if (c[0] != 0 || c[1] != 0 || c[2] != 0) return 0;
  int64_t t = dot3(w, d), dd = dot3(d, d);
  if (dd == 0) return w[0] == 0 && w[1] == 0 && w[2] == 0;
  return t >= 0 && t <= dd;
}

/* Is v in the closed triangle abc (a point set in R^3)?  Written with 3-D
 * cross products: v must be coplanar with abc and on the inner (or boundary)
 * side of every edge, measured against the triangle normal n.  A zero-area
 * triangle is the segment hull of its three corners. */
int32_t orc_point_in_closed_triangle(const int64_t *v, const int64_t *a,
                                     const int64_t *b, const int64_t *c) {
  int64_t ab[3], ac[3], n[3];
  sub3(b, a, ab);
  sub3(c, a, ac);
  cross3(ab, ac, n);
  if (n[0] == 0 && n[1] == 0 && n[2] == 0) {
    /* collinear or coincident corners: the hull is the longest of the three
     * segments between them */
    return on_closed_segment(v, a, b) || on_closed_segment(v, b, c) ||
           on_closed_segment(v, a, c);
  }
  int64_t av[3];
  sub3(v, a, av);
  if (dot3(av, n) != 0) return 0; /* < 2^18 * 2^37 * 3, fits */
  const int64_t *P[3] = {a, b, c};
  for (int k = 0; k < 3; ++k) {
    const int64_t *s = P[k], *e = P[(k + 1) % 3];
    int64_t se[3], sv[3], cr[3];
    sub3(e, s, se);
    sub3(v, s, sv);
    cross3(se, sv, cr);
    if (dot3_128(cr, n) < 0) return 0; /* 2^37 * 2^37 products: __int128 */
  }
  return 1;
}

/* Sign of orient2d_xy(a, b, v + (e, e^2)) for an infinitesimal e > 0.  The
 * exact value is o + (bx-ax) e^2 - (by-ay) e, with o = orient2d_xy(a,b,v). */
static int perturbed_side(const int64_t *a, const int64_t *b, const int64_t *v) {
  int64_t o = orc_orient2d_xy(a, b, v);
  if (o != 0) return sgn(o);
  if (a[1] != b[1]) return sgn(a[1] - b[1]);
  return sgn(b[0] - a[0]);
}

/* Does the +z ray from v (perturbed to (x+e, y+e^2)) hit triangle abc?
 * Requires: the triangle's xy projection has nonzero area, the perturbed
 * point lies strictly inside that projection, and v lies strictly below the
 * triangle's plane.  Below means orient3d(a,b,c,v) and the projected area
 * orient2d_xy(a,b,c) have opposite signs (orient3d = (v-a).n and n_z is the
 * projected area; the plane point above v is v + h z with h = -(v-a).n/n_z). */
int32_t orc_ray_up_hits(const int64_t *v, const int64_t *a, const int64_t *b,
                        const int64_t *c) {
  int s2 = sgn(orc_orient2d_xy(a, b, c));
  if (s2 == 0) return 0;
  if (perturbed_side(a, b, v) != s2) return 0;
  if (perturbed_side(b, c, v) != s2) return 0;
  if (perturbed_side(c, a, v) != s2) return 0;
  int s3 = sgn(orc_orient3d(a, b, c, v));
  return (s3 != 0 && s3 == -s2) ? 1 : 0;
}

/* ---------------------------------------------------------------------- */
/* Mesh conversion                                                          */
/* ---------------------------------------------------------------------- */

static void mesh_free(mesh_t *m) {
  free(m->v);
  free(m->t);
  m->v = NULL;
  m->t = NULL;
}

/* Convert mesh k of dataset D, translated by off (may be NULL). */
static int mesh_load(const orc_dataset *D, int64_t k, const int32_t *off,
                     mesh_t *m) {
  memset(m, 0, sizeof(*m));
  if (k < 0 || k >= D->nmesh) return ORC_ERR_ARG;
  int64_t v0 = D->voff[k], v1 = D->voff[k + 1];
  int64_t t0 = D->toff[k], t1 = D->toff[k + 1];
  m->nv = v1 - v0;
  m->nf = t1 - t0;
  m->v = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(m->nv > 0 ? m->nv : 1));
  m->t = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(m->nf > 0 ? m->nf : 1));
  if (!m->v || !m->t) { mesh_free(m); return ORC_ERR_NOMEM; }
  for (int d = 0; d < 3; ++d) { m->lo[d] = INT64_MAX; m->hi[d] = INT64_MIN; }
  for (int64_t i = 0; i < m->nv; ++i) {
    for (int d = 0; d < 3; ++d) {
      double f = (double)D->xyz[3 * (v0 + i) + d];
      int64_t q = (int64_t)f;
      if ((double)q != f) { mesh_free(m); return ORC_ERR_RANGE; }
      if (off) q += off[d];
      if (q < 0 || q >= ORC_GRID) { mesh_free(m); return ORC_ERR_RANGE; }
      m->v[3 * i + d] = q;
      if (q < m->lo[d]) m->lo[d] = q;
      if (q > m->hi[d]) m->hi[d] = q;
    }
  }
  for (int64_t i = 0; i < 3 * m->nf; ++i) {
    int32_t id = D->tris[3 * t0 + i];
    if (id < 0 || id >= m->nv) { mesh_free(m); return ORC_ERR_INDEX; }
    m->t[i] = id;
  }
  return ORC_OK;
}

#define VTX(m, i) (&(m)->v[3 * (int64_t)(i)])

/* ---------------------------------------------------------------------- */
/* cross(A,B)                                                              */
/* ---------------------------------------------------------------------- */

static int boxes_meet(const int64_t *lo0, const int64_t *hi0,
                      const int64_t *lo1, const int64_t *hi1) {
  for (int d = 0; d < 3; ++d)
    if (lo0[d] > hi1[d] || lo1[d] > hi0[d]) return 0;
  return 1;
}

static void seg_box(const int64_t *p, const int64_t *q, int64_t *lo, int64_t *hi) {
  for (int d = 0; d < 3; ++d) {
    lo[d] = p[d] < q[d] ? p[d] : q[d];
    hi[d] = p[d] < q[d] ? q[d] : p[d];
  }
}
static void tri_box(const int64_t *a, const int64_t *b, const int64_t *c,
                    int64_t *lo, int64_t *hi) {
  for (int d = 0; d < 3; ++d) {
    int64_t l = a[d], h = a[d];
    if (b[d] < l) l = b[d];
    if (c[d] < l) l = c[d];
    if (b[d] > h) h = b[d];
    if (c[d] > h) h = c[d];
    lo[d] = l;
    hi[d] = h;
  }
}

/* Does some edge of S pierce some triangle of T?  tier 2 restricts the tests
 * to edges and triangles whose boxes meet the clip box [clo, chi] and each
 * other (the triangles meeting the clip box are listed once per call). */
static int pierce_one_way(const mesh_t *S, const mesh_t *T, int tier,
                          const int64_t *clo, const int64_t *chi,
                          int64_t *ntests) {
  int64_t *list = NULL, nlist = T->nf;
  if (tier == 2) {
    list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T->nf > 0 ? T->nf : 1));
    if (!list) return ORC_ERR_NOMEM;
    nlist = 0;
    for (int64_t g = 0; g < T->nf; ++g) {
      int64_t tlo[3], thi[3];
      tri_box(VTX(T, T->t[3 * g]), VTX(T, T->t[3 * g + 1]), VTX(T, T->t[3 * g + 2]), tlo, thi);
      if (boxes_meet(tlo, thi, clo, chi)) list[nlist++] = g;
    }
  }
  int found = 0;
  for (int64_t f = 0; f < S->nf && !found; ++f) {
    for (int k = 0; k < 3 && !found; ++k) {
      const int64_t *p = VTX(S, S->t[3 * f + k]);
      const int64_t *q = VTX(S, S->t[3 * f + (k + 1) % 3]);
      int64_t slo[3], shi[3];
      if (tier == 2) {
        seg_box(p, q, slo, shi);
        if (!boxes_meet(slo, shi, clo, chi)) continue;
      }
      for (int64_t h = 0; h < nlist; ++h) {
        int64_t g = tier == 2 ? list[h] : h;
        const int64_t *a = VTX(T, T->t[3 * g]);
        const int64_t *b = VTX(T, T->t[3 * g + 1]);
        const int64_t *c = VTX(T, T->t[3 * g + 2]);
        if (tier == 2) {
          int64_t tlo[3], thi[3];
          tri_box(a, b, c, tlo, thi);
          if (!boxes_meet(tlo, thi, slo, shi)) continue;
        }
        ++*ntests;
        if (orc_segtri_strict(p, q, a, b, c)) { found = 1; break; }
      }
    }
  }
  free(list);
  return found;
}

static int cross_meshes(const mesh_t *A, const mesh_t *B, int tier,
                        int64_t *ntests) {
  int64_t clo[3], chi[3];
  for (int d = 0; d < 3; ++d) {
    clo[d] = A->lo[d] > B->lo[d] ? A->lo[d] : B->lo[d];
    chi[d] = A->hi[d] < B->hi[d] ? A->hi[d] : B->hi[d];
    if (tier == 2 && clo[d] > chi[d]) return 0;
  }
  int r = pierce_one_way(A, B, tier, clo, chi, ntests);
  if (r != 0) return r;
  return pierce_one_way(B, A, tier, clo, chi, ntests);
}

/* ---------------------------------------------------------------------- */
/* inside(B,A)                                                             */
/* ---------------------------------------------------------------------- */

static int on_surface(const int64_t *v, const mesh_t *A) {
  for (int64_t g = 0; g < A->nf; ++g) {
    if (orc_point_in_closed_triangle(v, VTX(A, A->t[3 * g]),
                                     VTX(A, A->t[3 * g + 1]),
                                     VTX(A, A->t[3 * g + 2])))
      return 1;
  }
  return 0;
}

static int parity_up(const int64_t *v, const mesh_t *A) {
  int par = 0;
  for (int64_t g = 0; g < A->nf; ++g)
    par ^= orc_ray_up_hits(v, VTX(A, A->t[3 * g]), VTX(A, A->t[3 * g + 1]),
                           VTX(A, A->t[3 * g + 2]));
  return par;
}

/* qsort has no context argument; one per thread, so that several threads may
 * refine disjoint candidate lists at once (every other object is per call) */
static _Thread_local const mesh_t *g_sort_mesh;
static int lex_cmp(const void *x, const void *y) {
  const int64_t *p = VTX(g_sort_mesh, *(const int64_t *)x);
  const int64_t *q = VTX(g_sort_mesh, *(const int64_t *)y);
  for (int d = 0; d < 3; ++d) {
    if (p[d] < q[d]) return -1;
    if (p[d] > q[d]) return 1;
  }
  int64_t i = *(const int64_t *)x, j = *(const int64_t *)y;
  return (i > j) - (i < j);
}

/* Index of the lexicographically smallest vertex of B not on the closed
 * surface of A, or -1 if every vertex of B lies on A's surface. */
static int64_t rep_vertex(const mesh_t *B, const mesh_t *A) {
  if (B->nv == 0) return -1;
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)B->nv);
  if (!order) return -2;
  for (int64_t i = 0; i < B->nv; ++i) order[i] = i;
  g_sort_mesh = B;
  qsort(order, (size_t)B->nv, sizeof(int64_t), lex_cmp);
  int64_t rep = -1;
  for (int64_t k = 0; k < B->nv; ++k) {
    if (!on_surface(VTX(B, order[k]), A)) { rep = order[k]; break; }
  }
  free(order);
  return rep;
}

static int inside_meshes(const mesh_t *B, const mesh_t *A, int64_t *nparity) {
  int64_t r = rep_vertex(B, A);
  if (r < 0) return r == -2 ? ORC_ERR_NOMEM : 0; /* -1: no representative */
  ++*nparity;
  return parity_up(VTX(B, r), A);
}

/* ---------------------------------------------------------------------- */
/* Exported pair and join functions                                        */
/* ---------------------------------------------------------------------- */

/* stats[0] += segment/triangle tests, stats[1] += parity rays cast. */
static int pair_eval(const orc_dataset *DA, int64_t i, const orc_dataset *DB,
                     int64_t j, const int32_t *off, int tier, int what,
                     int64_t *stats) {
  mesh_t A, B;
  int rc = mesh_load(DA, i, NULL, &A);
  if (rc) return rc;
  rc = mesh_load(DB, j, off, &B);
  if (rc) { mesh_free(&A); return rc; }
  int64_t dummy[2] = {0, 0};
  if (!stats) stats = dummy;
  int res = 0;
  /* what: 1 = cross, 2 = inside(B,A), 4 = inside(A,B); any set bit -> OR */
  if (what & 1) res = cross_meshes(&A, &B, tier, &stats[0]);
  if (!res && (what & 2)) {
    rc = inside_meshes(&B, &A, &stats[1]);
    if (rc < 0) res = rc; else res = rc;
  }
  if (!res && (what & 4)) {
    rc = inside_meshes(&A, &B, &stats[1]);
    if (rc < 0) res = rc; else res = rc;
  }
  mesh_free(&A);
  mesh_free(&B);
  return res;
}

/* intersects(A_i, B_j [+ off]) -> 1/0, or a negative error code. */
int32_t orc_intersects_pair(const orc_dataset *DA, int64_t i,
                            const orc_dataset *DB, int64_t j,
                            const int32_t *off, int32_t tier, int64_t *stats) {
  return pair_eval(DA, i, DB, j, off, tier, 7, stats);
}

/* The three sub-predicates separately, for tests. */
int32_t orc_cross_pair(const orc_dataset *DA, int64_t i, const orc_dataset *DB,
                       int64_t j, int32_t tier) {
  return pair_eval(DA, i, DB, j, NULL, tier, 1, NULL);
}
int32_t orc_inside_pair(const orc_dataset *DB, int64_t j,
                        const orc_dataset *DA, int64_t i) {
  /* inside(B_j, A_i): note the argument order (B first) */
  return pair_eval(DA, i, DB, j, NULL, 1, 2, NULL);
}

/* The paper's three join predicates for one pair (A_i, B_j [+ off]):
 *   ORC_PRED_INTERSECTS  cross OR inside(B,A) OR inside(A,B)          (Sec. 3.4)
 *   ORC_PRED_OVERLAP     cross: a surface crossing, bidirectional     (Sec. 3.2)
 *   ORC_PRED_CONTAINS    A_i contains B_j: no crossing, and B_j's
 *                        representative vertex inside A_i    (Sec. 3.3, Alg. 2)
 *   ORC_PRED_WITHIN      A_i within B_j, i.e. B_j contains A_i: the role swap
 *                        of the containment test                     (Sec. 3.3)
 *   ORC_PRED_ANY_VERTEX  intersects, or some vertex of either mesh strictly
 *                        inside the other: a completeness mode for the
 *                        strict rule's blind spot (surfaces that cross only
 *                        through edge and vertex coincidences); still sound,
 *                        since such a vertex is an interior point of the other
 *                        solid on the boundary of its own
 * As in Alg. 2 the crossing test runs first and only a pair without a
 * crossing gets the parity test.  Returns 1/0 or a negative error code. */
enum { ORC_PRED_INTERSECTS = 0, ORC_PRED_OVERLAP = 1, ORC_PRED_CONTAINS = 2,
       ORC_PRED_WITHIN = 3, ORC_PRED_ANY_VERTEX = 4 };

/* Some vertex of B lies strictly inside A (off A's surface, odd parity). */
static int any_vertex_inside(const mesh_t *B, const mesh_t *A, int64_t *nparity) {
  for (int64_t k = 0; k < B->nv; ++k) {
    const int64_t *v = VTX(B, k);
    if (on_surface(v, A)) continue;
    ++*nparity;
    if (parity_up(v, A)) return 1;
  }
  return 0;
}

static int pair_pred(const orc_dataset *DA, int64_t i, const orc_dataset *DB,
                     int64_t j, const int32_t *off, int tier, int pred,
                     int64_t *stats) {
  if (pred == ORC_PRED_INTERSECTS) return pair_eval(DA, i, DB, j, off, tier, 7, stats);
  if (pred == ORC_PRED_ANY_VERTEX) {
    int r = pair_eval(DA, i, DB, j, off, tier, 7, stats);
    if (r != 0) return r;
  } else if (pred != ORC_PRED_OVERLAP && pred != ORC_PRED_CONTAINS &&
             pred != ORC_PRED_WITHIN) {
    return ORC_ERR_ARG;
  }
  mesh_t A, B;
  int rc = mesh_load(DA, i, NULL, &A);
  if (rc) return rc;
  rc = mesh_load(DB, j, off, &B);
  if (rc) { mesh_free(&A); return rc; }
  int64_t dummy[2] = {0, 0};
  if (!stats) stats = dummy;
  int res;
  if (pred == ORC_PRED_ANY_VERTEX) {
    res = any_vertex_inside(&B, &A, &stats[1]);
    if (!res) res = any_vertex_inside(&A, &B, &stats[1]);
    mesh_free(&A);
    mesh_free(&B);
    return res;
  }
  res = cross_meshes(&A, &B, tier, &stats[0]);
  if (res >= 0 && pred != ORC_PRED_OVERLAP) {
    if (res) res = 0;                                   /* a crossing pair */
    else if (pred == ORC_PRED_CONTAINS) res = inside_meshes(&B, &A, &stats[1]);
    else res = inside_meshes(&A, &B, &stats[1]);
  }
  mesh_free(&A);
  mesh_free(&B);
  return res;
}

/* orc_join with a predicate (ORC_PRED_*): flags[c] for candidate c. */
int64_t orc_join_pred(const orc_dataset *DA, const orc_dataset *DB,
                      const int32_t *cand, const int32_t *off, int64_t n,
                      int32_t tier, int32_t pred, uint8_t *flags, int64_t *stats) {
  int64_t k = 0;
  for (int64_t c = 0; c < n; ++c) {
    int r = pair_pred(DA, cand[2 * c], DB, cand[2 * c + 1], off ? off + 3 * c : NULL,
                      tier, pred, stats);
    if (r < 0) return r;
    flags[c] = (uint8_t)r;
    k += r;
  }
  return k;
}

/* Representative vertex of B_j with respect to A_i (mesh-local index, or -1). */
int64_t orc_rep_vertex(const orc_dataset *DB, int64_t j, const orc_dataset *DA,
                       int64_t i) {
  mesh_t A, B;
  int rc = mesh_load(DA, i, NULL, &A);
  if (rc) return rc;
  rc = mesh_load(DB, j, NULL, &B);
  if (rc) { mesh_free(&A); return rc; }
  int64_t r = rep_vertex(&B, &A);
  mesh_free(&A);
  mesh_free(&B);
  return r;
}

/* Parity of the +z ray from the integer point v against mesh A_i, and whether
 * v lies on A_i's closed surface (bit 1 of the result). */
int32_t orc_point_query(const int64_t *v, const orc_dataset *DA, int64_t i) {
  mesh_t A;
  int rc = mesh_load(DA, i, NULL, &A);
  if (rc) return rc;
  int r = parity_up(v, &A) | (on_surface(v, &A) << 1);
  mesh_free(&A);
  return r;
}

/* Refine candidate pairs.  cand: n x 2 (i, j); off: n x 3 translations of
 * B_j per candidate, or NULL.  flags: n bytes out.  stats: 2 counters (may be
 * NULL).  Returns the number of intersecting pairs or a negative error. */
int64_t orc_join(const orc_dataset *DA, const orc_dataset *DB,
                 const int32_t *cand, const int32_t *off, int64_t n,
                 int32_t tier, uint8_t *flags, int64_t *stats) {
  int64_t k = 0;
  for (int64_t c = 0; c < n; ++c) {
    int r = orc_intersects_pair(DA, cand[2 * c], DB, cand[2 * c + 1],
                                off ? off + 3 * c : NULL, tier, stats);
    if (r < 0) return r;
    flags[c] = (uint8_t)r;
    k += r;
  }
  return k;
}

/* Candidate pairs whose closed mesh bounding boxes meet, in (i, j)
 * lexicographic order; self != 0 keeps i < j only.  Writes at most cap pairs,
 * returns the total count (or a negative error). */
int64_t orc_mbb_candidates(const orc_dataset *DA, const orc_dataset *DB,
                           int32_t self, int32_t *out, int64_t cap) {
  int64_t na = DA->nmesh, nb = DB->nmesh;
  int64_t *box = (int64_t *)malloc(sizeof(int64_t) * 6 * (size_t)(na + nb + 1));
  if (!box) return ORC_ERR_NOMEM;
  for (int s = 0; s < 2; ++s) {
    const orc_dataset *D = s ? DB : DA;
    for (int64_t m = 0; m < D->nmesh; ++m) {
      int64_t *b = box + 6 * (s ? na + m : m);
      for (int d = 0; d < 3; ++d) { b[d] = INT64_MAX; b[3 + d] = INT64_MIN; }
      for (int64_t v = D->voff[m]; v < D->voff[m + 1]; ++v)
        for (int d = 0; d < 3; ++d) {
          double f = (double)D->xyz[3 * v + d];
          int64_t q = (int64_t)f;
          if ((double)q != f || q < 0 || q >= ORC_GRID) { free(box); return ORC_ERR_RANGE; }
          if (q < b[d]) b[d] = q;
          if (q > b[3 + d]) b[3 + d] = q;
        }
    }
  }
  int64_t k = 0;
  for (int64_t i = 0; i < na; ++i)
    for (int64_t j = self ? i + 1 : 0; j < nb; ++j) {
      const int64_t *x = box + 6 * i, *y = box + 6 * (na + j);
      if (boxes_meet(x, x + 3, y, y + 3)) {
        if (k < cap) { out[2 * k] = (int32_t)i; out[2 * k + 1] = (int32_t)j; }
        ++k;
      }
    }
  free(box);
  return k;
}

/* Closed-manifold check of mesh k: every undirected edge is used by exactly
 * two triangles and no triangle repeats a vertex.  Returns 1 if it holds. */
static int edge_cmp(const void *x, const void *y) {
  const int64_t *p = (const int64_t *)x, *q = (const int64_t *)y;
  if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
  if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
  return 0;
}
int32_t orc_is_closed_manifold(const orc_dataset *D, int64_t k) {
  int64_t t0 = D->toff[k], nf = D->toff[k + 1] - t0;
  int64_t nv = D->voff[k + 1] - D->voff[k];
  if (nf == 0) return 0;
  int64_t *e = (int64_t *)malloc(sizeof(int64_t) * 6 * (size_t)nf);
  if (!e) return ORC_ERR_NOMEM;
  for (int64_t f = 0; f < nf; ++f) {
    for (int j = 0; j < 3; ++j) {
      int64_t a = D->tris[3 * (t0 + f) + j], b = D->tris[3 * (t0 + f) + (j + 1) % 3];
      if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) { free(e); return 0; }
      e[2 * (3 * f + j)] = a < b ? a : b;
      e[2 * (3 * f + j) + 1] = a < b ? b : a;
    }
  }
  qsort(e, (size_t)(3 * nf), 2 * sizeof(int64_t), edge_cmp);
  int ok = 1;
  for (int64_t s = 0; s < 3 * nf && ok;) {
    int64_t r = s;
    while (r < 3 * nf && edge_cmp(e + 2 * r, e + 2 * s) == 0) ++r;
    if (r - s != 2) ok = 0;
    s = r;
  }
  free(e);
  return ok;
}
