/*
 * Independent FP64 CPU oracle for the occlusion-tested irradiance matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or constant with the
 * CUDA library and is deliberately plain: every segment is tested against
 * every triangle (brute force), in double precision; a CPU-BVH mode
 * (uvco_irradiance_bvh) gives the same results faster, for larger samples.
 *
 * What it computes (paper Sec. IV-C, "Discrete Radiative Fluence"):
 *
 *   For candidate i, lamp source m and patch j:
 *     o   = fl32(c_i + off_m)       source point: the FP32 sum, so that both
 *                                   sides start from the same point
 *     v   = o - s_j                 from the patch point to the source
 *     d   = |v|,  cos = <n_j, v>/d  (n_j points into the free space)
 *     V   = 1 iff cos > 0 and no triangle other than the patch's own (excl)
 *           meets the open segment {o + tau (s_j - o) : 0 < tau < 1}
 *           (visibility rule stated under Eq. (7))
 *     E_ij = sum_m  w_m P <v, n_j> / (4 pi d^3) * V       (Eq. (7), with the
 *           printed cases read the other way round: the formula applies when
 *           the patch is visible, zero otherwise; w_m P is the power of
 *           source m, equal shares for a line lamp, Sec. IV-C "Non-Point
 *           Light Sources")
 *
 *   Grazing flags (pairs where an FP32 implementation may legitimately
 *   disagree on V); eps is an absolute distance in metres, OR-ed over the
 *   facing sources of the pair:
 *     bit 0  the closed segment [o, s_j] passes within eps of an edge of a
 *            non-excluded triangle
 *     bit 1  an endpoint (o or s_j) lies within eps of a non-excluded triangle
 *     bit 2  |<n_j, v>| <= eps (the facing decision is within eps of flipping)
 *
 *   The flag tests skip a triangle only when that is exact: a segment whose
 *   endpoints are both farther than eps from the triangle's plane on the same
 *   side, or whose distance to the triangle's bounding sphere exceeds eps,
 *   cannot come within eps of the triangle.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double x, y, z; } d3;

static d3 v3(double x, double y, double z) { d3 r = {x, y, z}; return r; }
static d3 vsub(d3 a, d3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static d3 vadd(d3 a, d3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static d3 vmul(d3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static double vdot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static d3 vcross(d3 a, d3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double vnorm(d3 a) { return sqrt(vdot(a, a)); }
static double clamp01(double t) { return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t); }

/* Does the open segment o + tau*dir, 0 < tau < 1, meet the closed triangle
 * (a,b,c)?  Moller-Trumbore in FP64: solve o + tau dir = a + u e1 + w e2. */
static int segment_meets_triangle(d3 o, d3 dir, d3 a, d3 b, d3 c) {
    d3 e1 = vsub(b, a), e2 = vsub(c, a);
    d3 p = vcross(dir, e2);
    double det = vdot(e1, p);
    if (det == 0.0) return 0;            /* segment parallel to the plane */
    d3 r = vsub(o, a);
    double u = vdot(r, p) / det;
    if (u < 0.0 || u > 1.0) return 0;
    d3 q = vcross(r, e1);
    double w = vdot(dir, q) / det;
    if (w < 0.0 || u + w > 1.0) return 0;
    double tau = vdot(e2, q) / det;
    return tau > 0.0 && tau < 1.0;
}

/* Distance between closed segments [p1,q1] and [p2,q2]: minimise
 * |p1 + s d1 - p2 - t d2| over s,t in [0,1] (clamp the unconstrained optimum
 * of one parameter, solve for the other, re-clamp). */
static double segment_segment_distance(d3 p1, d3 q1, d3 p2, d3 q2) {
    d3 d1 = vsub(q1, p1), d2 = vsub(q2, p2), r = vsub(p1, p2);
    double a = vdot(d1, d1), e = vdot(d2, d2), f = vdot(d2, r);
    double s, t;
    if (a == 0.0 && e == 0.0) return vnorm(r);
    if (a == 0.0) {
        s = 0.0;
        t = clamp01(f / e);
    } else {
        double c = vdot(d1, r);
        if (e == 0.0) {
            t = 0.0;
            s = clamp01(-c / a);
        } else {
            double b = vdot(d1, d2);
            double den = a * e - b * b;
            s = den > 0.0 ? clamp01((b * f - c * e) / den) : 0.0;
            t = (b * s + f) / e;
            if (t < 0.0) {
                t = 0.0;
                s = clamp01(-c / a);
            } else if (t > 1.0) {
                t = 1.0;
                s = clamp01((b - c) / a);
            }
        }
    }
    return vnorm(vsub(vadd(p1, vmul(d1, s)), vadd(p2, vmul(d2, t))));
}

static double point_segment_distance(d3 p, d3 a, d3 b) {
    d3 ab = vsub(b, a);
    double L = vdot(ab, ab);
    double t = L > 0.0 ? clamp01(vdot(vsub(p, a), ab) / L) : 0.0;
    return vnorm(vsub(p, vadd(a, vmul(ab, t))));
}

static double point_triangle_distance(d3 p, d3 a, d3 b, d3 c) {
    d3 n = vcross(vsub(b, a), vsub(c, a));
    double nn = vdot(n, n);
    double de = fmin(point_segment_distance(p, a, b),
                     fmin(point_segment_distance(p, b, c), point_segment_distance(p, c, a)));
    if (nn == 0.0) return de;
    double h = vdot(vsub(p, a), n) / nn;
    d3 pp = vsub(p, vmul(n, h));          /* projection onto the plane */
    int inside = vdot(vcross(vsub(b, a), vsub(pp, a)), n) >= 0.0 &&
                 vdot(vcross(vsub(c, b), vsub(pp, b)), n) >= 0.0 &&
                 vdot(vcross(vsub(a, c), vsub(pp, c)), n) >= 0.0;
    return inside ? fabs(h) * sqrt(nn) : de;
}

typedef struct {
    d3 a, b, c;        /* vertices */
    d3 n;              /* unit plane normal (zero for degenerate triangles) */
    d3 center;         /* bounding-sphere centre (vertex mean) */
    double radius;     /* bounding-sphere radius */
} tri64;

static int build_tris(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, tri64* T) {
    for (int64_t t = 0; t < nt; ++t) {
        int32_t ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
        if (ia < 0 || ib < 0 || ic < 0 || ia >= nv || ib >= nv || ic >= nv) return -1;
        T[t].a = v3(verts[3 * ia], verts[3 * ia + 1], verts[3 * ia + 2]);
        T[t].b = v3(verts[3 * ib], verts[3 * ib + 1], verts[3 * ib + 2]);
        T[t].c = v3(verts[3 * ic], verts[3 * ic + 1], verts[3 * ic + 2]);
        d3 n = vcross(vsub(T[t].b, T[t].a), vsub(T[t].c, T[t].a));
        double nl = vnorm(n);
        T[t].n = nl > 0.0 ? vmul(n, 1.0 / nl) : v3(0, 0, 0);
        T[t].center = vmul(vadd(vadd(T[t].a, T[t].b), T[t].c), 1.0 / 3.0);
        T[t].radius = fmax(vnorm(vsub(T[t].a, T[t].center)),
                           fmax(vnorm(vsub(T[t].b, T[t].center)), vnorm(vsub(T[t].c, T[t].center))));
    }
    return 0;
}

/* Grazing test of the closed segment [o,s] against one triangle (bits 0,1). */
static int grazing_bits(const tri64* t, d3 o, d3 s, double eps) {
    /* exact skip 1: both endpoints farther than eps from the plane, same side */
    if (t->n.x != 0.0 || t->n.y != 0.0 || t->n.z != 0.0) {
        double da = vdot(vsub(o, t->a), t->n), db = vdot(vsub(s, t->a), t->n);
        if ((da > eps && db > eps) || (da < -eps && db < -eps)) return 0;
    }
    /* exact skip 2: segment farther than eps from the bounding sphere */
    if (point_segment_distance(t->center, o, s) > t->radius + eps) return 0;
    int bits = 0;
    if (segment_segment_distance(o, s, t->a, t->b) <= eps ||
        segment_segment_distance(o, s, t->b, t->c) <= eps ||
        segment_segment_distance(o, s, t->c, t->a) <= eps)
        bits |= 1;
    if (point_triangle_distance(o, t->a, t->b, t->c) <= eps ||
        point_triangle_distance(s, t->a, t->b, t->c) <= eps)
        bits |= 2;
    return bits;
}

/*
 * CPU-BVH mode.  A binary bounding-volume hierarchy over the triangles (boxes
 * from the FP64 vertices, exact; median split of the triangle centres along
 * the widest axis; leaves of at most 4 triangles) restricts each segment's
 * triangle tests to the triangles whose box, padded by `pad`, the closed
 * segment crosses.  The tests themselves are the brute force's
 * (segment_meets_triangle, grazing_bits), so the mode gives the same entries,
 * bits and flags whenever the box test never rejects a triangle the brute
 * force would count: a segment point inside a triangle lies inside its box,
 * and the padding (1e-9 of the scene's diagonal, plus eps for the flags) is
 * far above the rounding of the FP64 slab test.
 */
typedef struct {
    double lo[3], hi[3];
    int64_t left, right;   /* children, or -1 for a leaf */
    int64_t first, count;  /* leaf: order[first .. first+count) */
} bnode;

typedef struct {
    bnode* nodes;
    int64_t* order;
    int64_t nnodes;
    double diag;
} bvh64;

typedef struct { double key; int64_t idx; } keyed;

static int keyed_cmp(const void* a, const void* b) {
    const keyed* x = (const keyed*)a;
    const keyed* y = (const keyed*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static void box_of(const tri64* T, const int64_t* order, int64_t first, int64_t count, double lo[3], double hi[3]) {
    for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t q = first; q < first + count; ++q) {
        const tri64* t = &T[order[q]];
        const d3 v[3] = {t->a, t->b, t->c};
        for (int e = 0; e < 3; ++e) {
            const double c[3] = {v[e].x, v[e].y, v[e].z};
            for (int k = 0; k < 3; ++k) {
                if (c[k] < lo[k]) lo[k] = c[k];
                if (c[k] > hi[k]) hi[k] = c[k];
            }
        }
    }
}

static void bvh_free(bvh64* B) {
    free(B->nodes);
    free(B->order);
    B->nodes = NULL;
    B->order = NULL;
}

static int bvh_build(const tri64* T, int64_t nt, bvh64* B) {
    B->nnodes = 0;
    B->nodes = (bnode*)malloc(sizeof(bnode) * (size_t)(2 * (nt > 0 ? nt : 1)));
    B->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
    keyed* tmp = (keyed*)malloc(sizeof(keyed) * (size_t)(nt > 0 ? nt : 1));
    int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * (nt > 0 ? nt : 1)));
    if (!B->nodes || !B->order || !tmp || !stack) { free(tmp); free(stack); bvh_free(B); return -2; }
    for (int64_t t = 0; t < nt; ++t) B->order[t] = t;
    B->diag = 0.0;
    if (nt == 0) { free(tmp); free(stack); return 0; }
    bnode* root = &B->nodes[B->nnodes++];
    root->first = 0;
    root->count = nt;
    box_of(T, B->order, 0, nt, root->lo, root->hi);
    B->diag = sqrt((root->hi[0] - root->lo[0]) * (root->hi[0] - root->lo[0]) +
                   (root->hi[1] - root->lo[1]) * (root->hi[1] - root->lo[1]) +
                   (root->hi[2] - root->lo[2]) * (root->hi[2] - root->lo[2]));
    int64_t top = 0;
    stack[top++] = 0;
    while (top > 0) {
        bnode* nd = &B->nodes[stack[--top]];
        nd->left = nd->right = -1;
        if (nd->count <= 4) continue;
        double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t q = nd->first; q < nd->first + nd->count; ++q) {
            const d3 c = T[B->order[q]].center;
            const double cc[3] = {c.x, c.y, c.z};
            for (int k = 0; k < 3; ++k) {
                if (cc[k] < clo[k]) clo[k] = cc[k];
                if (cc[k] > chi[k]) chi[k] = cc[k];
            }
        }
        int axis = 0;
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
        for (int64_t q = 0; q < nd->count; ++q) {
            const d3 c = T[B->order[nd->first + q]].center;
            tmp[q].key = axis == 0 ? c.x : (axis == 1 ? c.y : c.z);
            tmp[q].idx = B->order[nd->first + q];
        }
        qsort(tmp, (size_t)nd->count, sizeof(keyed), keyed_cmp);
        for (int64_t q = 0; q < nd->count; ++q) B->order[nd->first + q] = tmp[q].idx;
        const int64_t half = nd->count / 2;
        const int64_t li = B->nnodes++, ri = B->nnodes++;
        bnode* L = &B->nodes[li];
        bnode* R = &B->nodes[ri];
        L->first = nd->first;
        L->count = half;
        R->first = nd->first + half;
        R->count = nd->count - half;
        box_of(T, B->order, L->first, L->count, L->lo, L->hi);
        box_of(T, B->order, R->first, R->count, R->lo, R->hi);
        nd->left = li;
        nd->right = ri;
        stack[top++] = li;
        stack[top++] = ri;
    }
    free(tmp);
    free(stack);
    return 0;
}

/* Does the closed segment o + tau dir, 0 <= tau <= 1, meet the box padded by pad? */
static int segment_meets_box(d3 o, d3 dir, const double lo[3], const double hi[3], double pad) {
    const double oo[3] = {o.x, o.y, o.z}, dd[3] = {dir.x, dir.y, dir.z};
    double t0 = 0.0, t1 = 1.0;
    for (int k = 0; k < 3; ++k) {
        const double l = lo[k] - pad, h = hi[k] + pad;
        if (dd[k] == 0.0) {
            if (oo[k] < l || oo[k] > h) return 0;
            continue;
        }
        double ta = (l - oo[k]) / dd[k], tb = (h - oo[k]) / dd[k];
        if (ta > tb) { const double x = ta; ta = tb; tb = x; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* Visibility of the open segment o -> o + dir through the hierarchy (any hit). */
static int bvh_visible(const bvh64* B, const tri64* T, int32_t ex0, int32_t ex1, d3 o, d3 dir, int64_t* stack) {
    if (B->nnodes == 0) return 1;
    const double pad = 1e-9 * B->diag + 1e-300;
    int64_t top = 0;
    stack[top++] = 0;
    while (top > 0) {
        const bnode* nd = &B->nodes[stack[--top]];
        if (!segment_meets_box(o, dir, nd->lo, nd->hi, pad)) continue;
        if (nd->left < 0) {
            for (int64_t q = nd->first; q < nd->first + nd->count; ++q) {
                const int64_t t = B->order[q];
                if (t == ex0 || t == ex1) continue;
                if (segment_meets_triangle(o, dir, T[t].a, T[t].b, T[t].c)) return 0;
            }
        } else {
            stack[top++] = nd->left;
            stack[top++] = nd->right;
        }
    }
    return 1;
}

/* Grazing bits 0 and 1 of the closed segment [o, s] through the hierarchy. */
static int bvh_grazing(const bvh64* B, const tri64* T, int32_t ex0, int32_t ex1, d3 o, d3 s, double eps,
                       int64_t* stack) {
    if (B->nnodes == 0) return 0;
    const double pad = eps + 1e-9 * B->diag + 1e-300;
    const d3 dir = vsub(s, o);
    int bits = 0;
    int64_t top = 0;
    stack[top++] = 0;
    while (top > 0 && bits != 3) {
        const bnode* nd = &B->nodes[stack[--top]];
        if (!segment_meets_box(o, dir, nd->lo, nd->hi, pad)) continue;
        if (nd->left < 0) {
            for (int64_t q = nd->first; q < nd->first + nd->count; ++q) {
                const int64_t t = B->order[q];
                if (t == ex0 || t == ex1) continue;
                bits |= grazing_bits(&T[t], o, s, eps);
            }
        } else {
            stack[top++] = nd->left;
            stack[top++] = nd->right;
        }
    }
    return bits;
}

/*
 * Irradiance entries for a list of (candidate, patch) pairs; with B non-NULL
 * the segment and flag tests go through the hierarchy (same results).
 *   pairs    npairs*2 int64 (i, j); NULL means every pair, i major (k = i*np + j)
 *   E_out    npairs doubles (W/m^2)
 *   vis_out  npairs*K bytes (1 = source m sees the patch point), may be NULL
 *   flag_out npairs bytes of grazing bits, may be NULL (then no flag work)
 * Returns 0, or -1 on an index out of range.
 */
static int irradiance_entries(const tri64* T, int64_t nt, const bvh64* B, const float* centroid,
                              const float* normal, const int32_t* excl, int64_t np, const float* cand,
                              const float* offsets, const float* weights, int32_t K, double power,
                              const int64_t* pairs, int64_t npairs, double eps, double* E_out, uint8_t* vis_out,
                              uint8_t* flag_out, int nthreads) {
    const double four_pi = 4.0 * M_PI;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int64_t* stack = B ? (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * B->nnodes + 2)) : NULL;
        if (B && !stack) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
        for (int64_t k = 0; k < npairs; ++k) {
            if (B && !stack) continue;
            int64_t i = pairs ? pairs[2 * k] : k / np;
            int64_t j = pairs ? pairs[2 * k + 1] : k % np;
            d3 s = v3(centroid[3 * j], centroid[3 * j + 1], centroid[3 * j + 2]);
            d3 n = v3(normal[3 * j], normal[3 * j + 1], normal[3 * j + 2]);
            int32_t ex0 = excl[2 * j], ex1 = excl[2 * j + 1];
            double E = 0.0;
            int flags = 0;
            for (int m = 0; m < K; ++m) {
                /* the source point in FP32 (one IEEE single add per coordinate) */
                float ox = cand[3 * i] + offsets[3 * m];
                float oy = cand[3 * i + 1] + offsets[3 * m + 1];
                float oz = cand[3 * i + 2] + offsets[3 * m + 2];
                d3 o = v3(ox, oy, oz);
                d3 v = vsub(o, s);
                double d = vnorm(v);
                double nv_ = vdot(n, v);
                int visible = 0;
                if (flag_out && fabs(nv_) <= eps) flags |= 4;
                if (nv_ > 0.0 && d > 0.0) {
                    d3 dir = vsub(s, o);
                    if (B) {
                        visible = bvh_visible(B, T, ex0, ex1, o, dir, stack);
                        if (flag_out) flags |= bvh_grazing(B, T, ex0, ex1, o, s, eps, stack);
                    } else {
                        visible = 1;
                        for (int64_t t = 0; t < nt; ++t) {
                            if (t == ex0 || t == ex1) continue;
                            if (segment_meets_triangle(o, dir, T[t].a, T[t].b, T[t].c)) { visible = 0; break; }
                        }
                        if (flag_out)
                            for (int64_t t = 0; t < nt; ++t) {
                                if (t == ex0 || t == ex1) continue;
                                flags |= grazing_bits(&T[t], o, s, eps);
                            }
                    }
                    if (visible) E += (double)weights[m] * power * nv_ / (four_pi * d * d * d);
                }
                if (vis_out) vis_out[k * K + m] = (uint8_t)visible;
            }
            E_out[k] = E;
            if (flag_out) flag_out[k] = (uint8_t)flags;
        }
        free(stack);
    }
    return failed ? -2 : 0;
}

static int check_irradiance_args(const int32_t* excl, int64_t np, int64_t nc, int64_t nt, int32_t K,
                                 const int64_t* pairs, int64_t npairs) {
    if (K < 1 || nt < 0 || np < 0 || nc < 0) return -1;
    for (int64_t j = 0; j < np; ++j)
        for (int q = 0; q < 2; ++q)
            if (excl[2 * j + q] < -1 || excl[2 * j + q] >= nt) return -1;
    if (pairs != NULL)
        for (int64_t k = 0; k < npairs; ++k)
            if (pairs[2 * k] < 0 || pairs[2 * k] >= nc || pairs[2 * k + 1] < 0 || pairs[2 * k + 1] >= np)
                return -1;
    return 0;
}

/* Brute force: every segment against every triangle. */
int uvco_irradiance(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                    const float* centroid, const float* normal, const int32_t* excl, int64_t np,
                    const float* cand, int64_t nc,
                    const float* offsets, const float* weights, int32_t K, double power,
                    const int64_t* pairs, int64_t npairs, double eps,
                    double* E_out, uint8_t* vis_out, uint8_t* flag_out, int nthreads) {
    if (pairs == NULL) npairs = nc * np;
    if (check_irradiance_args(excl, np, nc, nt, K, pairs, npairs) != 0) return -1;
    tri64* T = (tri64*)malloc(sizeof(tri64) * (size_t)(nt > 0 ? nt : 1));
    if (!T) return -2;
    if (build_tris(verts, nv, tris, nt, T) != 0) { free(T); return -1; }
    int rc = irradiance_entries(T, nt, NULL, centroid, normal, excl, np, cand, offsets, weights, K, power, pairs,
                                npairs, eps, E_out, vis_out, flag_out, nthreads);
    free(T);
    return rc;
}

/* The same entries through the CPU hierarchy (see bvh_build). */
int uvco_irradiance_bvh(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                        const float* centroid, const float* normal, const int32_t* excl, int64_t np,
                        const float* cand, int64_t nc,
                        const float* offsets, const float* weights, int32_t K, double power,
                        const int64_t* pairs, int64_t npairs, double eps,
                        double* E_out, uint8_t* vis_out, uint8_t* flag_out, int nthreads) {
    if (pairs == NULL) npairs = nc * np;
    if (check_irradiance_args(excl, np, nc, nt, K, pairs, npairs) != 0) return -1;
    tri64* T = (tri64*)malloc(sizeof(tri64) * (size_t)(nt > 0 ? nt : 1));
    if (!T) return -2;
    if (build_tris(verts, nv, tris, nt, T) != 0) { free(T); return -1; }
    bvh64 B;
    int rc = bvh_build(T, nt, &B);
    if (rc == 0) {
        rc = irradiance_entries(T, nt, &B, centroid, normal, excl, np, cand, offsets, weights, K, power, pairs,
                                npairs, eps, E_out, vis_out, flag_out, nthreads);
        bvh_free(&B);
    }
    free(T);
    return rc;
}

/* Number of threads an OpenMP region will use (1 without OpenMP). */
int uvco_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Solid angle of triangle (a, b, c) seen from o, by van Oosterom and
 * Strackee (IEEE Trans. Biomed. Eng. 30(2), 1983):
 *   tan(Omega / 2) = |R1 . (R2 x R3)| /
 *                    (r1 r2 r3 + (R1.R2) r3 + (R1.R3) r2 + (R2.R3) r1)
 * with R_k the vectors from o to the vertices and r_k their lengths; the
 * numerator is evaluated as R1 . ((b - a) x (c - a)), the same value.
 */
static double solid_angle(d3 o, d3 a, d3 b, d3 c) {
    d3 R1 = vsub(a, o), R2 = vsub(b, o), R3 = vsub(c, o);
    double r1 = vnorm(R1), r2 = vnorm(R2), r3 = vnorm(R3);
    double num = fabs(vdot(R1, vcross(vsub(b, a), vsub(c, a))));
    double den = r1 * r2 * r3 + vdot(R1, R2) * r3 + vdot(R1, R3) * r2 + vdot(R2, R3) * r1;
    return 2.0 * atan2(num, den);
}

static int segment_visible(const tri64* T, int64_t nt, int32_t ex0, int32_t ex1, d3 o, d3 p) {
    d3 dir = vsub(p, o);
    for (int64_t t = 0; t < nt; ++t) {
        if (t == ex0 || t == ex1) continue;
        if (segment_meets_triangle(o, dir, T[t].a, T[t].b, T[t].c)) return 0;
    }
    return 1;
}

static int segment_grazing(const tri64* T, int64_t nt, int32_t ex0, int32_t ex1, d3 o, d3 p, double eps) {
    int bits = 0;
    for (int64_t t = 0; t < nt; ++t) {
        if (t == ex0 || t == ex1) continue;
        bits |= grazing_bits(&T[t], o, p, eps);
    }
    return bits;
}

/* Visibility and grazing bits of one segment o -> p, brute force or through the hierarchy. */
static int seg_visible(const tri64* T, int64_t nt, const bvh64* B, int64_t* stack, int32_t ex0, int32_t ex1, d3 o,
                       d3 p) {
    return B ? bvh_visible(B, T, ex0, ex1, o, vsub(p, o), stack) : segment_visible(T, nt, ex0, ex1, o, p);
}
static int seg_grazing(const tri64* T, int64_t nt, const bvh64* B, int64_t* stack, int32_t ex0, int32_t ex1, d3 o,
                       d3 p, double eps) {
    return B ? bvh_grazing(B, T, ex0, ex1, o, p, eps, stack) : segment_grazing(T, nt, ex0, ex1, o, p, eps);
}

/*
 * Area-mean irradiance of patches with known geometry (the mean of Eq. (4)
 * over the patch instead of its centroid sample): the flux a triangle
 * receives from an isotropic point source of power P that sees all of it is
 * P Omega / (4 pi), Omega its solid angle (the integral of cos / d^2 over
 * the triangle), so the patch's mean irradiance is P sum_t Omega_t / (4 pi a_j).
 *
 * Per candidate i, source m, patch j with triangles ptri[j][0..1] (the second
 * unused when its area is zero):
 *   o        = fl32(c_i + off_m)
 *   facing   <n_j, o - s_j> > 0 (centroid s_j)
 *   checks   the open segments from o to s_j and to each vertex q pulled
 *            towards the centroid, q' = fl32(q + fl32(delta * fl32(s_j - q)))
 *            (single-precision operations, no contraction)
 *   all visible      E += w_m P sum_t Omega_t(o) / (4 pi a_j)     (closed form)
 *   centroid visible E += w_m P <n_j, v> / (4 pi d^3)             (point sample)
 *   nclosed_out[k]   number of sources that used the closed form
 *   flag_out[k]      grazing bits (as above) OR-ed over every check segment
 *                    of the facing sources
 * With B non-NULL every check segment goes through the hierarchy (same results).
 * Returns 0, or -1 on an index out of range.
 */
static int area_mean_entries(const tri64* T, int64_t nt, const bvh64* B, const float* centroid, const float* normal,
                             const float* area, const int32_t* excl, const float* ptri, int64_t np,
                             const float* cand, const float* offsets, const float* weights, int32_t K,
                             double power, float delta, const int64_t* pairs, int64_t npairs, double eps,
                             double* E_out, uint8_t* nclosed_out, uint8_t* flag_out, int nthreads) {
    const double four_pi = 4.0 * M_PI;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int64_t* stack = B ? (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * B->nnodes + 2)) : NULL;
        if (B && !stack) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
        for (int64_t k = 0; k < npairs; ++k) {
            if (B && !stack) continue;
            int64_t i = pairs ? pairs[2 * k] : k / np;
            int64_t j = pairs ? pairs[2 * k + 1] : k % np;
            const float* sf = centroid + 3 * j;
            d3 s = v3(sf[0], sf[1], sf[2]);
            d3 n = v3(normal[3 * j], normal[3 * j + 1], normal[3 * j + 2]);
            int32_t ex0 = excl[2 * j], ex1 = excl[2 * j + 1];
            /* the patch triangles and the pulled-in check points */
            d3 tv[2][3];
            int ntri = 0;
            d3 chk[6];
            int nchk = 0;
            for (int t = 0; t < 2; ++t) {
                const float* g = ptri + 18 * j + 9 * t;
                for (int q = 0; q < 3; ++q) tv[t][q] = v3(g[3 * q], g[3 * q + 1], g[3 * q + 2]);
                d3 cr = vcross(vsub(tv[t][1], tv[t][0]), vsub(tv[t][2], tv[t][0]));
                if (vdot(cr, cr) == 0.0) continue;
                if (t != ntri)
                    for (int q = 0; q < 3; ++q) tv[ntri][q] = tv[t][q];
                for (int q = 0; q < 3; ++q) {
                    const float* gq = g + 3 * q;
                    float px = gq[0] + delta * (sf[0] - gq[0]);
                    float py = gq[1] + delta * (sf[1] - gq[1]);
                    float pz = gq[2] + delta * (sf[2] - gq[2]);
                    chk[nchk++] = v3(px, py, pz);
                }
                ++ntri;
            }
            double E = 0.0;
            int flags = 0, nclosed = 0;
            for (int m = 0; m < K; ++m) {
                float ox = cand[3 * i] + offsets[3 * m];
                float oy = cand[3 * i + 1] + offsets[3 * m + 1];
                float oz = cand[3 * i + 2] + offsets[3 * m + 2];
                d3 o = v3(ox, oy, oz);
                d3 v = vsub(o, s);
                double d = vnorm(v);
                double nv_ = vdot(n, v);
                if (flag_out && fabs(nv_) <= eps) flags |= 4;
                if (!(nv_ > 0.0 && d > 0.0)) continue;
                int vis_c = seg_visible(T, nt, B, stack, ex0, ex1, o, s);
                if (flag_out) flags |= seg_grazing(T, nt, B, stack, ex0, ex1, o, s, eps);
                int all = vis_c && ntri > 0;
                for (int q = 0; q < nchk; ++q) {
                    if (all && !seg_visible(T, nt, B, stack, ex0, ex1, o, chk[q])) all = 0;
                    if (flag_out && vis_c) flags |= seg_grazing(T, nt, B, stack, ex0, ex1, o, chk[q], eps);
                }
                double pw = (double)weights[m] * power;
                if (all) {
                    double om = 0.0;
                    for (int t = 0; t < ntri; ++t) om += solid_angle(o, tv[t][0], tv[t][1], tv[t][2]);
                    E += pw * om / (four_pi * (double)area[j]);
                    ++nclosed;
                } else if (vis_c) {
                    E += pw * nv_ / (four_pi * d * d * d);
                }
            }
            E_out[k] = E;
            if (nclosed_out) nclosed_out[k] = (uint8_t)nclosed;
            if (flag_out) flag_out[k] = (uint8_t)flags;
        }
        free(stack);
    }
    return failed ? -2 : 0;
}

static int area_mean_impl(int use_bvh, const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                          const float* centroid, const float* normal, const float* area, const int32_t* excl,
                          const float* ptri, int64_t np, const float* cand, int64_t nc, const float* offsets,
                          const float* weights, int32_t K, double power, float delta, const int64_t* pairs,
                          int64_t npairs, double eps, double* E_out, uint8_t* nclosed_out, uint8_t* flag_out,
                          int nthreads) {
    if (pairs == NULL) npairs = nc * np;
    if (check_irradiance_args(excl, np, nc, nt, K, pairs, npairs) != 0) return -1;
    tri64* T = (tri64*)malloc(sizeof(tri64) * (size_t)(nt > 0 ? nt : 1));
    if (!T) return -2;
    if (build_tris(verts, nv, tris, nt, T) != 0) { free(T); return -1; }
    int rc = 0;
    if (use_bvh) {
        bvh64 B;
        rc = bvh_build(T, nt, &B);
        if (rc == 0) {
            rc = area_mean_entries(T, nt, &B, centroid, normal, area, excl, ptri, np, cand, offsets, weights, K,
                                   power, delta, pairs, npairs, eps, E_out, nclosed_out, flag_out, nthreads);
            bvh_free(&B);
        }
    } else {
        rc = area_mean_entries(T, nt, NULL, centroid, normal, area, excl, ptri, np, cand, offsets, weights, K, power,
                               delta, pairs, npairs, eps, E_out, nclosed_out, flag_out, nthreads);
    }
    free(T);
    return rc;
}

int uvco_area_mean(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                   const float* centroid, const float* normal, const float* area, const int32_t* excl,
                   const float* ptri, int64_t np, const float* cand, int64_t nc,
                   const float* offsets, const float* weights, int32_t K, double power, float delta,
                   const int64_t* pairs, int64_t npairs, double eps,
                   double* E_out, uint8_t* nclosed_out, uint8_t* flag_out, int nthreads) {
    return area_mean_impl(0, verts, nv, tris, nt, centroid, normal, area, excl, ptri, np, cand, nc, offsets, weights,
                          K, power, delta, pairs, npairs, eps, E_out, nclosed_out, flag_out, nthreads);
}

/* The same area-mean entries through the CPU hierarchy (see bvh_build). */
int uvco_area_mean_bvh(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                       const float* centroid, const float* normal, const float* area, const int32_t* excl,
                       const float* ptri, int64_t np, const float* cand, int64_t nc,
                       const float* offsets, const float* weights, int32_t K, double power, float delta,
                       const int64_t* pairs, int64_t npairs, double eps,
                       double* E_out, uint8_t* nclosed_out, uint8_t* flag_out, int nthreads) {
    return area_mean_impl(1, verts, nv, tris, nt, centroid, normal, area, excl, ptri, np, cand, nc, offsets, weights,
                          K, power, delta, pairs, npairs, eps, E_out, nclosed_out, flag_out, nthreads);
}

/*
 * Visibility-cube estimator of the paper (Sec. IV-C, Fig. 2), by ray casting
 * through every pixel centre instead of rasterising.  Around each source point
 * o a cube of six R x R faces; face f looks along axis a = f / 2 with sign
 * s = +1 for even f, -1 for odd f; its pixel (px, py) is the direction
 *   dir[a] = s,  dir[(a+1) % 3] = u,  dir[(a+2) % 3] = v,
 *   u = fl32(fl32(2 px + 1) / R) - 1,  v = fl32(fl32(2 py + 1) / R) - 1
 * (single-precision operations, as the library forms them) and covers the
 * solid angle of the square [2px/R - 1, 2(px+1)/R - 1] x [2py/R - 1, ...] of
 * the plane at unit distance, Omega = G(u1,v1) - G(u0,v1) - G(u1,v0) + G(u0,v0)
 * with G(u, v) = atan(u v / sqrt(1 + u^2 + v^2)).  T = the nearest triangle
 * met by the ray o + t dir, t > 0; the pixel's power w_m P Omega / (4 pi)
 * goes to T when the ray meets T's front side (<dir, n_T> < 0) and is
 * absorbed otherwise.  F_out[i][t] sums it over the sources of candidate i
 * (flux, W); the mean irradiance is F / |s_t|.
 *
 * amb_out[i][t] bounds how much flux an FP32 implementation may legitimately
 * move to or from triangle t: a pixel whose ray passes within rel * t of the
 * boundary of a triangle not behind the nearest robust hit, or whose nearest
 * triangle is met within rel of edge-on, adds its power to every triangle
 * that could receive it.
 */
static double pixel_G(double u, double v) { return atan(u * v / sqrt(1.0 + u * u + v * v)); }

/* Could the pixel ray o + t dir (t > 0, |dir| = dl) reach triangle T within
 * the rounding an FP32 rasteriser may make?  tmax: the farthest parameter a
 * receiver may have (just beyond the nearest robust hit, or past the whole
 * scene when there is none).  A triangle the ray's line crosses is near when
 * the crossing point, at parameter tt in (0, tmax], lies within rel * tt * dl
 * of it; a triangle met edge-on (the ray parallel to its plane, det = 0) is
 * near when the stretch of the ray from o to parameter tmax passes within
 * rel * tmax * dl of it (distance of that segment from the triangle's edges
 * and of its end points from the triangle). */
static int raster_receiver(const tri64* T, d3 o, d3 dir, double dl, double tmax, double rel) {
    d3 e1 = vsub(T->b, T->a), e2 = vsub(T->c, T->a);
    d3 p = vcross(dir, e2);
    double det = vdot(e1, p);
    if (det == 0.0) {
        d3 q = vadd(o, vmul(dir, tmax));
        double dist = fmin(point_triangle_distance(o, T->a, T->b, T->c),
                           point_triangle_distance(q, T->a, T->b, T->c));
        dist = fmin(dist, segment_segment_distance(o, q, T->a, T->b));
        dist = fmin(dist, segment_segment_distance(o, q, T->b, T->c));
        dist = fmin(dist, segment_segment_distance(o, q, T->c, T->a));
        return dist <= rel * tmax * dl;
    }
    d3 r = vsub(o, T->a);
    d3 qq = vcross(r, e1);
    double tt = vdot(e2, qq) / det;
    if (!(tt > 0.0) || tt > tmax) return 0;
    d3 h = vadd(o, vmul(dir, tt));
    return point_triangle_distance(h, T->a, T->b, T->c) <= rel * tt * dl;
}

int uvco_raster(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const float* tri_normal,
                const float* cand, int64_t nc, const float* offsets, const float* weights, int32_t K, double power,
                int32_t R, double rel, double* F_out, double* amb_out, int nthreads) {
    if (K < 1 || nt < 0 || nc < 0 || R < 1) return -1;
    tri64* T = (tri64*)malloc(sizeof(tri64) * (size_t)(nt > 0 ? nt : 1));
    if (!T) return -2;
    if (build_tris(verts, nv, tris, nt, T) != 0) { free(T); return -1; }
    for (int64_t k = 0; k < nc * nt; ++k) { F_out[k] = 0.0; if (amb_out) amb_out[k] = 0.0; }
    const int64_t npix = 6 * (int64_t)R * R;
    /* bounding box of the triangles: a ray that meets nothing robustly is
     * followed to the far side of the scene when looking for receivers */
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = 0; t < nt; ++t) {
        const d3 w[3] = {T[t].a, T[t].b, T[t].c};
        for (int k = 0; k < 3; ++k) {
            lo[0] = fmin(lo[0], w[k].x); hi[0] = fmax(hi[0], w[k].x);
            lo[1] = fmin(lo[1], w[k].y); hi[1] = fmax(hi[1], w[k].y);
            lo[2] = fmin(lo[2], w[k].z); hi[2] = fmax(hi[2], w[k].z);
        }
    }
    const d3 mid = v3(0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2]));
    const double radius = nt > 0 ? 0.5 * vnorm(v3(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2])) : 0.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int64_t i = 0; i < nc; ++i)
        for (int m = 0; m < K; ++m) {
            float ox = cand[3 * i] + offsets[3 * m];
            float oy = cand[3 * i + 1] + offsets[3 * m + 1];
            float oz = cand[3 * i + 2] + offsets[3 * m + 2];
            d3 o = v3(ox, oy, oz);
            double pw = (double)weights[m] * power / (4.0 * M_PI);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
            for (int64_t q = 0; q < npix; ++q) {
                int f = (int)(q / ((int64_t)R * R));
                int px = (int)(q % ((int64_t)R * R)) % R, py = (int)(q % ((int64_t)R * R)) / R;
                int a = f / 2;
                double s = (f % 2 == 0) ? 1.0 : -1.0;
                float uf = (float)(2 * px + 1) / (float)R - 1.0f;
                float vf = (float)(2 * py + 1) / (float)R - 1.0f;
                double dd[3];
                dd[a] = s; dd[(a + 1) % 3] = uf; dd[(a + 2) % 3] = vf;
                d3 dir = v3(dd[0], dd[1], dd[2]);
                double dl = vnorm(dir);
                double u0 = 2.0 * px / R - 1.0, u1 = 2.0 * (px + 1) / R - 1.0;
                double v0 = 2.0 * py / R - 1.0, v1 = 2.0 * (py + 1) / R - 1.0;
                double e = pw * (pixel_G(u1, v1) - pixel_G(u0, v1) - pixel_G(u1, v0) + pixel_G(u0, v0));
                /* nearest hit, nearest robust hit, and the near candidates */
                int64_t best = -1;
                double tbest = INFINITY, trob = INFINITY;
                for (int64_t t = 0; t < nt; ++t) {
                    d3 e1 = vsub(T[t].b, T[t].a), e2 = vsub(T[t].c, T[t].a);
                    d3 p = vcross(dir, e2);
                    double det = vdot(e1, p);
                    if (det == 0.0) continue;
                    d3 r = vsub(o, T[t].a);
                    double uu = vdot(r, p) / det;
                    d3 qq = vcross(r, e1);
                    double ww = vdot(dir, qq) / det;
                    double tt = vdot(e2, qq) / det;
                    if (!(tt > 0.0)) continue;
                    int inside = uu >= 0.0 && ww >= 0.0 && uu + ww <= 1.0;
                    if (inside && tt < tbest) { tbest = tt; best = t; }
                    if (inside) {
                        d3 h = vadd(o, vmul(dir, tt));
                        double sd = fmin(point_segment_distance(h, T[t].a, T[t].b),
                                         fmin(point_segment_distance(h, T[t].b, T[t].c),
                                              point_segment_distance(h, T[t].c, T[t].a)));
                        if (sd > rel * tt * dl && tt < trob) trob = tt;
                    }
                }
                if (best >= 0) {
                    d3 nb = v3(tri_normal[3 * best], tri_normal[3 * best + 1], tri_normal[3 * best + 2]);
                    double dn = vdot(dir, nb);
                    if (dn < 0.0) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                        F_out[i * nt + best] += e;
                    }
                    if (amb_out && fabs(dn) <= rel * dl * vnorm(nb)) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                        amb_out[i * nt + best] += e;
                    }
                }
                if (!amb_out) continue;
                /* receivers: inside or near, and not behind the nearest robust
                 * hit; every one of them gets the pixel's power when there are
                 * at least two (a first pass counts them, a second adds) */
                const double tmax = isfinite(trob) ? trob * (1.0 + rel) : (vnorm(vsub(o, mid)) + radius) / dl;
                int nrec = 0;
                for (int64_t t = 0; t < nt && nrec < 2; ++t)
                    if (raster_receiver(&T[t], o, dir, dl, tmax, rel)) ++nrec;
                if (nrec >= 2)
                    for (int64_t t = 0; t < nt; ++t)
                        if (raster_receiver(&T[t], o, dir, dl, tmax, rel)) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                            amb_out[i * nt + t] += e;
                        }
            }
        }
    free(T);
    return 0;
}
