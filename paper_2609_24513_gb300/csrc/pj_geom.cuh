// Device geometry for the refinement kernels: exact orientation signs on the
// 2^18 integer grid (FP32 filter with a per-test error bound, int64 fallback),
// the strict segment/triangle test, the perturbed +z parity ray, the closed
// point-on-triangle test and a conservative segment/box slab test.
//
// Paper: the edge ray of Sec. 3.1 Step I (origin v_a, extent |v_b - v_a|) is
// kept as the unnormalised segment p + t (q - p), t in [0, 1]; a hit in
// Step II is decided by the exact sign pattern of five orientations instead
// of an FP32 ray/triangle distance, which makes the watertightness the
// paper gets from its ray tracer (Sec. 3.6 "Robustness") exact.
#pragma once
#include <stdint.h>

namespace pj {

struct F3 {
  float x, y, z;
};
struct I3 {
  int x, y, z;
};

__device__ __forceinline__ F3 mkf3(float x, float y, float z) {
  F3 r;
  r.x = x;
  r.y = y;
  r.z = z;
  return r;
}
__device__ __forceinline__ F3 sub(F3 a, F3 b) {
  // exact: both operands are integers below 2^19 in magnitude
  return mkf3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}
__device__ __forceinline__ F3 add(F3 a, F3 b) {
  return mkf3(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z));
}
__device__ __forceinline__ I3 toi(F3 a) {
  I3 r;
  r.x = __float2int_rn(a.x);
  r.y = __float2int_rn(a.y);
  r.z = __float2int_rn(a.z);
  return r;
}

__device__ __forceinline__ F3 ld3(const float *p) { return mkf3(p[0], p[1], p[2]); }

struct Box {
  F3 lo, hi;
};

// The parity ray leaves along the axis and direction with the shortest way out
// of the target's box (see ray_axis_hit: the parity does not depend on it).
__device__ __forceinline__ void ray_axis_choice(F3 v, F3 lo, F3 hi, int &ax, int &dir) {
  float best = hi.z - v.z;
  ax = 2;
  dir = 1;
  const float d[6] = {hi.x - v.x, v.x - lo.x, hi.y - v.y, v.y - lo.y, hi.z - v.z, v.z - lo.z};
  for (int k = 0; k < 6; ++k)
    if (d[k] < best) {
      best = d[k];
      ax = k >> 1;
      dir = (k & 1) ? -1 : 1;
    }
}

// does the ray (ax, dir) from v meet the closed box?
__device__ __forceinline__ bool ray_axis_box(F3 v, const Box &b, int ax, int dir) {
  const float vu = ax == 0 ? v.y : (ax == 1 ? v.z : v.x);
  const float vw = ax == 0 ? v.z : (ax == 1 ? v.x : v.y);
  const float lu = ax == 0 ? b.lo.y : (ax == 1 ? b.lo.z : b.lo.x);
  const float hu = ax == 0 ? b.hi.y : (ax == 1 ? b.hi.z : b.hi.x);
  const float lw = ax == 0 ? b.lo.z : (ax == 1 ? b.lo.x : b.lo.y);
  const float hw = ax == 0 ? b.hi.z : (ax == 1 ? b.hi.x : b.hi.y);
  const float va = ax == 0 ? v.x : (ax == 1 ? v.y : v.z);
  const float la = ax == 0 ? b.lo.x : (ax == 1 ? b.lo.y : b.lo.z);
  const float ha = ax == 0 ? b.hi.x : (ax == 1 ? b.hi.y : b.hi.z);
  return lu <= vu && vu <= hu && lw <= vw && vw <= hw && (dir > 0 ? va <= ha : la <= va);
}

// ---------------------------------------------------------------------------
// FP32 filter.
//
// A triple product x . (y x z) of exact FP32 integer vectors, evaluated as
// sum_i x_i * (y_j z_k - y_k z_j) with round-to-nearest and no contraction,
// differs from the exact value by at most about 5u * perm (u = 2^-24,
// perm = sum_i |x_i| (|y_j z_k| + |y_k z_j|)): 2u per minor, u per product
// with x_i, u per each of the two additions.  This is the stage-A argument of
// Shewchuk, "Adaptive Precision Floating-Point Arithmetic and Fast Robust
// Geometric Predicates" (1997), specialised to single precision.  The filter
// uses 8u = 2^-21 times the permanent computed in FP32, which covers the
// rounding of the permanent itself.  A sign is certified only when
// |det| > bound; everything else goes to the int64 path.
// ---------------------------------------------------------------------------
#define PJ_FILTER_COEF 4.76837158203125e-07f /* 2^-21 */

struct CrossP {
  F3 m;   // y x z (rounded)
  F3 pm;  // |y_j z_k| + |y_k z_j| per component (rounded)
};

__device__ __forceinline__ CrossP cross_p(F3 y, F3 z) {
  float p1 = __fmul_rn(y.y, z.z), p2 = __fmul_rn(y.z, z.y);
  float p3 = __fmul_rn(y.z, z.x), p4 = __fmul_rn(y.x, z.z);
  float p5 = __fmul_rn(y.x, z.y), p6 = __fmul_rn(y.y, z.x);
  CrossP c;
  c.m = mkf3(__fsub_rn(p1, p2), __fsub_rn(p3, p4), __fsub_rn(p5, p6));
  c.pm = mkf3(__fadd_rn(fabsf(p1), fabsf(p2)), __fadd_rn(fabsf(p3), fabsf(p4)),
              __fadd_rn(fabsf(p5), fabsf(p6)));
  return c;
}

// x . c.m and its error bound
__device__ __forceinline__ void dot_p(F3 x, const CrossP &c, float &det,
                                     float &err) {
  det = __fadd_rn(__fadd_rn(__fmul_rn(x.x, c.m.x), __fmul_rn(x.y, c.m.y)),
                  __fmul_rn(x.z, c.m.z));
  float perm =
      __fadd_rn(__fadd_rn(__fmul_rn(fabsf(x.x), c.pm.x),
                          __fmul_rn(fabsf(x.y), c.pm.y)),
                __fmul_rn(fabsf(x.z), c.pm.z));
  err = __fmul_rn(perm, PJ_FILTER_COEF);
}

// certified sign: +1 / -1, or 0 when the filter cannot decide
__device__ __forceinline__ int cert(float v, float e) {
  return v > e ? 1 : (v < -e ? -1 : 0);
}

// Orientations the filter cannot decide are most often exact zeros of a
// simple kind, which plain comparisons certify: four points in one
// axis-aligned plane (walls, floors and roofs of grid-aligned solids that
// touch) or a fourth point equal to one of the first three (shared
// vertices).  Either makes the determinant exactly 0, the value the int64
// path would compute.
__device__ __forceinline__ bool zero_orient(F3 a, F3 b, F3 c, F3 d) {
  return (a.x == b.x && b.x == c.x && c.x == d.x) || (a.y == b.y && b.y == c.y && c.y == d.y) ||
         (a.z == b.z && b.z == c.z && c.z == d.z) ||
         (d.x == a.x && d.y == a.y && d.z == a.z) || (d.x == b.x && d.y == b.y && d.z == b.z) ||
         (d.x == c.x && d.y == c.y && d.z == c.z);
}

// ---------------------------------------------------------------------------
// int64 orientation (exact).  Differences are below 2^19 in magnitude (grid
// 2^18, translated candidates stay on the grid), 2x2 minors below 2^39 and a
// triple product below 3 * 2^58.
// ---------------------------------------------------------------------------
struct L3 {
  long long x, y, z;
};
__device__ __forceinline__ L3 cross64(I3 a, I3 b) {
  L3 r;
  r.x = (long long)a.y * b.z - (long long)a.z * b.y;
  r.y = (long long)a.z * b.x - (long long)a.x * b.z;
  r.z = (long long)a.x * b.y - (long long)a.y * b.x;
  return r;
}
__device__ __forceinline__ long long dot64(I3 a, L3 b) {
  return (long long)a.x * b.x + (long long)a.y * b.y + (long long)a.z * b.z;
}
__device__ __forceinline__ I3 isub(I3 a, I3 b) {
  I3 r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  r.z = a.z - b.z;
  return r;
}
__device__ __forceinline__ int sgn64(long long v) { return (v > 0) - (v < 0); }

// Strict crossing from the exact signs.  With A = a - p, B = b - p,
// C = c - p, d = q - p:  orient(p,q,a,b) = d.(A x B), orient(p,q,b,c) =
// d.(B x C), orient(p,q,c,a) = d.(C x A), orient(a,b,c,p) = -A.(B x C) and
// orient(a,b,c,q) = -(a - q).((b - q) x (c - q)).  The segment crosses iff
// the last two have opposite nonzero signs and the first three one nonzero
// sign.
// Exact strict test with early exits: the plane side of p and q first (two
// orientations), the three edge orientations only if the plane separates
// them.
__device__ __forceinline__ bool segtri_exact_staged(F3 pf, F3 qf, F3 af, F3 bf, F3 cf) {
  I3 p = toi(pf), q = toi(qf);
  I3 A = isub(toi(af), p), B = isub(toi(bf), p), C = isub(toi(cf), p);
  L3 bc = cross64(B, C);
  const int a1 = -sgn64(dot64(A, bc));
  I3 Aq = isub(toi(af), q), Bq = isub(toi(bf), q), Cq = isub(toi(cf), q);
  const int a2 = -sgn64(dot64(Aq, cross64(Bq, Cq)));
  if (a1 == 0 || a2 == 0 || a1 == a2) return false;
  I3 d = isub(q, p);
  const int su = sgn64(dot64(d, cross64(A, B)));
  if (su == 0) return false;
  if (sgn64(dot64(d, bc)) != su) return false;
  return sgn64(dot64(d, cross64(C, A))) == su;
}

// Strict test deciding each of the five signs by the FP32 filter and only
// the uncertain ones in int64, stopping at the first sign that settles the
// answer.  *exact is set when any sign needed int64.
__device__ __forceinline__ bool segtri_filtered(F3 p, F3 q, F3 a, F3 b, F3 c, bool *exact) {
  const F3 A = sub(a, p), B = sub(b, p), C = sub(c, p);
  const CrossP bc = cross_p(B, C);
  float dv, ev;
  dot_p(A, bc, dv, ev);
  int sp = -cert(dv, ev);
  if (sp == 0) {
    if (zero_orient(a, b, c, p)) return false;
    *exact = true;
    const I3 pi = toi(p);
    sp = -sgn64(dot64(isub(toi(a), pi), cross64(isub(toi(b), pi), isub(toi(c), pi))));
    if (sp == 0) return false;
  }
  const F3 Aq = sub(a, q), Bq = sub(b, q), Cq = sub(c, q);
  const CrossP bcq = cross_p(Bq, Cq);
  dot_p(Aq, bcq, dv, ev);
  int sq = -cert(dv, ev);
  if (sq == 0) {
    if (zero_orient(a, b, c, q)) return false;
    *exact = true;
    const I3 qi = toi(q);
    sq = -sgn64(dot64(isub(toi(a), qi), cross64(isub(toi(b), qi), isub(toi(c), qi))));
  }
  if (sq == 0 || sq == sp) return false;
  const F3 d = sub(q, p);
  // u = d.(A x B), v = d.(B x C), w = d.(C x A): one sign, none zero
  int su;
  {
    const CrossP ab = cross_p(A, B);
    dot_p(d, ab, dv, ev);
    su = cert(dv, ev);
    if (su == 0) {
      if (zero_orient(p, q, a, b)) return false;
      *exact = true;
      const I3 pi = toi(p);
      su = sgn64(dot64(isub(toi(q), pi), cross64(isub(toi(a), pi), isub(toi(b), pi))));
      if (su == 0) return false;
    }
  }
  {
    dot_p(d, bc, dv, ev);
    int sv = cert(dv, ev);
    if (sv == -su) return false;
    if (sv == 0) {
      if (zero_orient(p, q, b, c)) return false;
      *exact = true;
      const I3 pi = toi(p);
      sv = sgn64(dot64(isub(toi(q), pi), cross64(isub(toi(b), pi), isub(toi(c), pi))));
      if (sv != su) return false;
    }
  }
  {
    const CrossP ca = cross_p(C, A);
    dot_p(d, ca, dv, ev);
    int sw = cert(dv, ev);
    if (sw == 0) {
      if (zero_orient(p, q, c, a)) return false;
      *exact = true;
      const I3 pi = toi(p);
      sw = sgn64(dot64(isub(toi(q), pi), cross64(isub(toi(c), pi), isub(toi(a), pi))));
    }
    return sw == su;
  }
}

// ---------------------------------------------------------------------------
// Segment / closed box slab test, conservative: never rejects a box that the
// exact closed segment meets.  Parameters t = (bound - p) / d use an exact
// difference and a correctly rounded reciprocal and product, so each has a
// relative error below 2^-22.9 and keeps its sign; comparing
// t_enter <= t_exit * (1 + 2^-20) absorbs it (cf. Ize, "Robust BVH Ray
// Traversal", JCGT 2013).  A zero direction component is decided exactly.
// The strict test with a static error bound: every point lies in a box of
// largest side D, so every difference of two points is at most D per
// coordinate, every permanent of the triple products at most 6 D^3, and
// the FP32 error at most 5u * 6 D^3 < 2^-18 D^3 (u = 2^-24); err = 2^-18 D^3
// (D^3 rounded upward far within the margin) certifies a sign with no
// per-test permanent.  Otherwise as segtri_filtered: simple exact zeros by
// comparison, the rest in int64.
__device__ __forceinline__ int cert_static(float det, float err) {
  return det > err ? 1 : (det < -err ? -1 : 0);
}
__device__ __forceinline__ float dot3(F3 x, F3 m) {
  return __fadd_rn(__fadd_rn(__fmul_rn(x.x, m.x), __fmul_rn(x.y, m.y)), __fmul_rn(x.z, m.z));
}
__device__ __forceinline__ F3 cross3(F3 y, F3 z) {
  return mkf3(__fsub_rn(__fmul_rn(y.y, z.z), __fmul_rn(y.z, z.y)),
              __fsub_rn(__fmul_rn(y.z, z.x), __fmul_rn(y.x, z.z)),
              __fsub_rn(__fmul_rn(y.x, z.y), __fmul_rn(y.y, z.x)));
}
__device__ __forceinline__ bool segtri_static_staged(F3 p, F3 q, F3 a, F3 b, F3 c, float err,
                                                    bool *exact) {
  const F3 A = sub(a, p), B = sub(b, p), C = sub(c, p);
  const F3 bc = cross3(B, C);
  int sp = -cert_static(dot3(A, bc), err);
  if (sp == 0) {
    if (zero_orient(a, b, c, p)) return false;
    *exact = true;
    const I3 pi = toi(p);
    sp = -sgn64(dot64(isub(toi(a), pi), cross64(isub(toi(b), pi), isub(toi(c), pi))));
    if (sp == 0) return false;
  }
  const F3 Aq = sub(a, q), Bq = sub(b, q), Cq = sub(c, q);
  int sq = -cert_static(dot3(Aq, cross3(Bq, Cq)), err);
  if (sq == 0) {
    if (zero_orient(a, b, c, q)) return false;
    *exact = true;
    const I3 qi = toi(q);
    sq = -sgn64(dot64(isub(toi(a), qi), cross64(isub(toi(b), qi), isub(toi(c), qi))));
  }
  if (sq == 0 || sq == sp) return false;
  const F3 d = sub(q, p);
  int su = cert_static(dot3(d, cross3(A, B)), err);
  if (su == 0) {
    if (zero_orient(p, q, a, b)) return false;
    *exact = true;
    const I3 pi = toi(p);
    su = sgn64(dot64(isub(toi(q), pi), cross64(isub(toi(a), pi), isub(toi(b), pi))));
    if (su == 0) return false;
  }
  int sv = cert_static(dot3(d, bc), err);
  if (sv == -su) return false;
  if (sv == 0) {
    if (zero_orient(p, q, b, c)) return false;
    *exact = true;
    const I3 pi = toi(p);
    sv = sgn64(dot64(isub(toi(q), pi), cross64(isub(toi(b), pi), isub(toi(c), pi))));
    if (sv != su) return false;
  }
  int sw = cert_static(dot3(d, cross3(C, A)), err);
  if (sw == 0) {
    if (zero_orient(p, q, c, a)) return false;
    *exact = true;
    const I3 pi = toi(p);
    sw = sgn64(dot64(isub(toi(q), pi), cross64(isub(toi(c), pi), isub(toi(a), pi))));
  }
  return sw == su;
}

// The same test with the five FP32 orientations evaluated together as
// independent chains (no early exit between them, so their latencies
// overlap).  Their certified signs settle the answer when the plane does not
// separate p and q, when two of u, v, w have opposite signs, or when all five
// are certified; any other pattern (some sign uncertain) goes through the
// staged test above, which decides the uncertain signs exactly.
__device__ __forceinline__ bool segtri_static(F3 p, F3 q, F3 a, F3 b, F3 c, float err,
                                             bool *exact) {
  const F3 A = sub(a, p), B = sub(b, p), C = sub(c, p);
  const F3 Aq = sub(a, q), Bq = sub(b, q), Cq = sub(c, q);
  const F3 d = sub(q, p);
  const F3 bc = cross3(B, C);
  const int sp = -cert_static(dot3(A, bc), err);
  const int sq = -cert_static(dot3(Aq, cross3(Bq, Cq)), err);
  const int su = cert_static(dot3(d, cross3(A, B)), err);
  const int sv = cert_static(dot3(d, bc), err);
  const int sw = cert_static(dot3(d, cross3(C, A)), err);
  if (sp != 0 && sp == sq) return false;                   // p, q on one side
  if (su * sv < 0 || sv * sw < 0 || su * sw < 0) return false;  // u, v, w disagree
  if (sp != 0 && sq != 0 && su != 0 && sv != 0 && sw != 0)
    return true;                                           // sp != sq, u = v = w
  return segtri_static_staged(p, q, a, b, c, err, exact);
}

// error bound of segtri_static for points in a box of largest side D:
// 2^-18 D^3, each product rounded upward
__device__ __forceinline__ float static_err(float D) {
  return __fmul_ru(__fmul_ru(__fmul_ru(D, D), D), 3.814697265625e-06f /* 2^-18 */);
}

// ---------------------------------------------------------------------------
struct Seg {
  F3 p;
  F3 inv;   // 1/d per axis (unused where d == 0)
  int zero; // bit k: d_k == 0
};

__device__ __forceinline__ Seg make_seg(F3 p, F3 q) {
  Seg s;
  s.p = p;
  F3 d = sub(q, p);
  s.zero = (d.x == 0.f) | ((d.y == 0.f) << 1) | ((d.z == 0.f) << 2);
  s.inv = mkf3(d.x == 0.f ? 0.f : __frcp_rn(d.x), d.y == 0.f ? 0.f : __frcp_rn(d.y),
               d.z == 0.f ? 0.f : __frcp_rn(d.z));
  return s;
}

__device__ __forceinline__ void slab_axis(float p, float inv, bool zero,
                                          float lo, float hi, float &tmin,
                                          float &tmax) {
  const float BIG = 1e30f;
  float t0, t1;
  if (zero) {
    t0 = (p >= lo) ? -BIG : BIG;
    t1 = (p <= hi) ? BIG : -BIG;
  } else {
    t0 = __fmul_rn(__fsub_rn(lo, p), inv);
    t1 = __fmul_rn(__fsub_rn(hi, p), inv);
  }
  tmin = fmaxf(tmin, fminf(t0, t1));
  tmax = fminf(tmax, fmaxf(t0, t1));
}

__device__ __forceinline__ bool slab_hit(const Seg &s, F3 lo, F3 hi) {
  float tmin = 0.f, tmax = 1.f;
  slab_axis(s.p.x, s.inv.x, s.zero & 1, lo.x, hi.x, tmin, tmax);
  slab_axis(s.p.y, s.inv.y, s.zero & 2, lo.y, hi.y, tmin, tmax);
  slab_axis(s.p.z, s.inv.z, s.zero & 4, lo.z, hi.z, tmin, tmax);
  return tmin <= __fmul_rn(tmax, 1.00000095367431640625f);  // 1 + 2^-20
}

// ---------------------------------------------------------------------------
// Parity ray (+z from v, perturbed to (x + e, y + e^2)) and point on a closed
// triangle.  All exact in int64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long o2xy(I3 a, I3 b, I3 c) {
  return (long long)(b.x - a.x) * (c.y - a.y) -
         (long long)(b.y - a.y) * (c.x - a.x);
}

// sign of orient2d_xy(a, b, v + (e, e^2)): the exact value plus the first
// nonvanishing coefficient of -(b_y - a_y) e + (b_x - a_x) e^2
__device__ __forceinline__ int side_eps(I3 a, I3 b, I3 v) {
  long long o = o2xy(a, b, v);
  if (o != 0) return sgn64(o);
  if (a.y != b.y) return a.y > b.y ? 1 : -1;
  return b.x > a.x ? 1 : (b.x < a.x ? -1 : 0);
}

// orient3d(a, b, c, v) = (v - a) . ((b - a) x (c - a))
__device__ __forceinline__ long long orient64(I3 a, I3 b, I3 c, I3 v) {
  return dot64(isub(v, a), cross64(isub(b, a), isub(c, a)));
}

__device__ __forceinline__ bool ray_up_hit(I3 v, I3 a, I3 b, I3 c) {
  long long s2 = o2xy(a, b, c);
  if (s2 == 0) return false;
  int s = s2 > 0 ? 1 : -1;
  if (side_eps(a, b, v) != s || side_eps(b, c, v) != s || side_eps(c, a, v) != s)
    return false;
  long long o = orient64(a, b, c, v);
  return o != 0 && sgn64(o) == -s;  // v strictly below the plane
}

// Parity ray from v along axis `ax` (0, 1, 2) in direction `dir` (+1 / -1).
// With (u, w, ax) a cyclic triple, v is perturbed to v + e u_hat + e^2 w_hat;
// the projected area orient2d_(u,w)(a,b,c) is the ax-component of the normal,
// and the plane point v + h e_ax has h = -orient3d(a,b,c,v) / n_ax, which must
// have the sign of dir.  For ax = 2, dir = +1 this is ray_up_hit.
//
// For a closed mod-2 cycle (every edge in exactly two triangles) and v off
// the surface, the parity of the hits is the mod-2 winding number of the
// surface around v, whichever axis and direction the ray takes: the perturbed
// origins all lie in v's component of the complement, and each perturbed ray
// crosses the surface only transversally through triangle interiors.
__device__ __forceinline__ int cget(I3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ bool ray_axis_hit(I3 v, I3 a, I3 b, I3 c, int ax, int dir) {
  const int u = ax == 2 ? 0 : ax + 1, w = ax == 0 ? 2 : ax - 1;
  I3 a2, b2, c2, v2;  // (u, w) coordinates in x, y
  a2.x = cget(a, u); a2.y = cget(a, w); a2.z = 0;
  b2.x = cget(b, u); b2.y = cget(b, w); b2.z = 0;
  c2.x = cget(c, u); c2.y = cget(c, w); c2.z = 0;
  v2.x = cget(v, u); v2.y = cget(v, w); v2.z = 0;
  long long s2 = o2xy(a2, b2, c2);
  if (s2 == 0) return false;
  int s = s2 > 0 ? 1 : -1;
  if (side_eps(a2, b2, v2) != s || side_eps(b2, c2, v2) != s || side_eps(c2, a2, v2) != s)
    return false;
  long long o = orient64(a, b, c, v);
  return o != 0 && sgn64(o) == -dir * s;
}

// 2-D closed point-in-triangle in the projection dropping axis `drop`
__device__ __forceinline__ bool in_tri_2d(I3 v, I3 a, I3 b, I3 c, int drop) {
  int ax, ay, bx, by, cx, cy, vx, vy;
  if (drop == 2) {
    ax = a.x; ay = a.y; bx = b.x; by = b.y; cx = c.x; cy = c.y; vx = v.x; vy = v.y;
  } else if (drop == 0) {
    ax = a.y; ay = a.z; bx = b.y; by = b.z; cx = c.y; cy = c.z; vx = v.y; vy = v.z;
  } else {
    ax = a.z; ay = a.x; bx = b.z; by = b.x; cx = c.z; cy = c.x; vx = v.z; vy = v.x;
  }
  long long area = (long long)(bx - ax) * (cy - ay) - (long long)(by - ay) * (cx - ax);
  long long e0 = (long long)(bx - ax) * (vy - ay) - (long long)(by - ay) * (vx - ax);
  long long e1 = (long long)(cx - bx) * (vy - by) - (long long)(cy - by) * (vx - bx);
  long long e2 = (long long)(ax - cx) * (vy - cy) - (long long)(ay - cy) * (vx - cx);
  if (area > 0) return e0 >= 0 && e1 >= 0 && e2 >= 0;
  return e0 <= 0 && e1 <= 0 && e2 <= 0;
}

// v on the segment hull of collinear points a, b, c
__device__ __forceinline__ bool on_collinear_hull(I3 v, I3 a, I3 b, I3 c) {
  int lx = min(a.x, min(b.x, c.x)), hx = max(a.x, max(b.x, c.x));
  int ly = min(a.y, min(b.y, c.y)), hy = max(a.y, max(b.y, c.y));
  int lz = min(a.z, min(b.z, c.z)), hz = max(a.z, max(b.z, c.z));
  if (v.x < lx || v.x > hx || v.y < ly || v.y > hy || v.z < lz || v.z > hz)
    return false;
  // a direction along the line: the two extreme corners of the box
  I3 p0 = a, p1 = (b.x != a.x || b.y != a.y || b.z != a.z) ? b : c;
  if (p1.x == p0.x && p1.y == p0.y && p1.z == p0.z) return true;  // single point
  L3 cr = cross64(isub(p1, p0), isub(v, p0));
  return cr.x == 0 && cr.y == 0 && cr.z == 0;
}

// v in the closed triangle abc (3-D point set)
__device__ __forceinline__ bool on_triangle(I3 v, I3 a, I3 b, I3 c) {
  L3 n = cross64(isub(b, a), isub(c, a));
  if (n.x == 0 && n.y == 0 && n.z == 0) return on_collinear_hull(v, a, b, c);
  if (dot64(isub(v, a), n) != 0) return false;
  long long ax = n.x < 0 ? -n.x : n.x, ay = n.y < 0 ? -n.y : n.y,
            az = n.z < 0 ? -n.z : n.z;
  int drop = (az >= ax && az >= ay) ? 2 : (ax >= ay ? 0 : 1);
  return in_tri_2d(v, a, b, c, drop);
}

}  // namespace pj
