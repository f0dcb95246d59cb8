/*
 * Counting replay of the irradiance kernels' wedge traversal (vertical line
 * lamps) on the CPU, for the memory roofline of the traversal.
 *
 * MEASUREMENT TOOL.  It is neither the oracle (it shares nothing with it and
 * checks nothing) nor the product: it re-executes, lane by lane and in FP32,
 * the visit order of the packet traversal over the four-wide hierarchy that
 * the library built (exported with uvc_scene_export_traversal), for a sample
 * of warp tasks, and counts what each warp and each lane loads.  The counts
 * give the algorithmic bytes per (candidate, patch) pair of the traversal
 * (paper Sec. IV-C: the visibility rule of Eq. (7), one segment per lamp
 * source of a line light):
 *
 *   per warp   bytes the memory system is asked for: one 128-byte node per
 *              node visit (the packet's loads are warp-uniform), 48 bytes
 *              per distinct triangle a leaf step of the warp loads, the
 *              cached occluder of each lane, the patch records (40 bytes per
 *              lane and task), and the output: 4 bytes of A and K bits of
 *              visibility per pair
 *   per lane   the same loads counted for every lane that needs them: 128
 *              bytes per node visit per searching lane, 48 bytes per leaf
 *              per lane
 *
 * Work unit (as in the kernels): a task is 32 consecutive patches (one per
 * lane) and a chunk of consecutive candidates; the lanes keep their patch
 * and their last occluder over the chunk.  Per candidate the K sources of
 * the vertical lamp are searched together: a wedge box test per child; the
 * leaf children a lane's wedge enters go to the warp's queue in lane order,
 * and every time 32 items wait the warp works off 32 of them (each with the
 * wanting lane's sources as they stood when the batch began: a plane test, a
 * lamp-height interval and the watertight segment test per remaining
 * source), then each lane drops the sources found occluded and narrows its
 * wedge; the items left when the traversal ends form a last batch.  The
 * arithmetic follows the kernels operation by operation (binary32, fused
 * multiply-adds where they fuse);
 * the approximate reciprocal of the height interval is taken exactly here,
 * so a source lying within rounding of an interval end may be counted
 * differently (the counts are compared with the kernels' own instrumented
 * counters in the tests).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXK 16
#define STACK 256

typedef struct {
    float q[6][4];
    int32_t r[4];
    int32_t m[4];
} node4_t;

typedef struct { float x, y, z, w; } f4;

typedef struct {
    const node4_t* nodes;
    const f4* tri;      /* [nt][3] */
    const f4* ps;
    const f4* pn;
    const int32_t* pe;  /* [np][2] */
    int64_t nt, np;
    int32_t root;
    float cut_eps;
} scene_t;

typedef struct {
    int K, wuniform;
    float oz[MAXK];
    float wz0, wrdz;
} lamp_t;

/* counters (per sample): see replay_counts */
enum {
    C_NODE_VISITS, C_LEAF_LOADS, C_TRAVERSALS, C_TRI_TESTS, C_SEARCH_SEGMENTS, C_BOX_TESTS, C_PLANE_TESTS,
    C_LEAF_STEPS, C_LEAF_STEP_LANES, C_LEAF_STEP_UNIQUE, C_CACHE_LOADS, C_LANE_NODE_VISITS, C_PAIRS, C_TASKS,
    C_NUM
};

static float fmax3(float a, float b, float c) { return fmaxf(fmaxf(a, b), c); }
static float fmin3(float a, float b, float c) { return fminf(fminf(a, b), c); }

static float safe_rcp(float d) {
    float a = fabsf(d) < 1e-30f ? copysignf(1e-30f, d) : d;
    return 1.0f / a;
}

static float pick(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

typedef struct { float sx, sy, sz; int kx, ky, kz; } shear_t;

/* set-up of the watertight test for direction (dx, dy, dz) */
static shear_t shear_of(float dx, float dy, float dz) {
    shear_t s;
    float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    int kz = ax > ay ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dkz = pick(dx, dy, dz, kz);
    if (dkz < 0.f) { int t = kx; kx = ky; ky = t; }
    s.kx = kx; s.ky = ky; s.kz = kz;
    s.sz = 1.0f / dkz;
    s.sx = pick(dx, dy, dz, kx) * s.sz;
    s.sy = pick(dx, dy, dz, ky) * s.sz;
    return s;
}

/* watertight segment/triangle test from (ox, oy, oz): hit iff the line
 * passes through the closed triangle and tau lies in (0, 1) */
static int seg_tri(float ox, float oy, float oz, const shear_t* h, const f4* a, const f4* b, const f4* c) {
    float Ax = a->x - ox, Ay = a->y - oy, Az = a->z - oz;
    float Bx = b->x - ox, By = b->y - oy, Bz = b->z - oz;
    float Cx = c->x - ox, Cy = c->y - oy, Cz = c->z - oz;
    float akz = pick(Ax, Ay, Az, h->kz), bkz = pick(Bx, By, Bz, h->kz), ckz = pick(Cx, Cy, Cz, h->kz);
    float ax = fmaf(-h->sx, akz, pick(Ax, Ay, Az, h->kx));
    float ay = fmaf(-h->sy, akz, pick(Ax, Ay, Az, h->ky));
    float bx = fmaf(-h->sx, bkz, pick(Bx, By, Bz, h->kx));
    float by = fmaf(-h->sy, bkz, pick(Bx, By, Bz, h->ky));
    float cx = fmaf(-h->sx, ckz, pick(Cx, Cy, Cz, h->kx));
    float cy = fmaf(-h->sy, ckz, pick(Cx, Cy, Cz, h->ky));
    float U = cx * by - cy * bx;
    float V = ax * cy - ay * cx;
    float W = bx * ay - by * ax;
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return 0;
    float det = U + V + W;
    if (det == 0.f) return 0;
    float pa = h->sz * akz, pb = h->sz * bkz, pc = h->sz * ckz;
    float T = fmaf(W, pc, fmaf(U, pa, V * pb));
    uint32_t ub, ud;
    memcpy(&ud, &det, 4);
    memcpy(&ub, &T, 4);
    uint32_t sgn = ud & 0x80000000u;
    ub ^= sgn;
    ud ^= sgn;
    float Ts, ds;
    memcpy(&Ts, &ub, 4);
    memcpy(&ds, &ud, 4);
    return Ts > 0.f && Ts < ds;
}

/* terms of one source against the patch point: v = o - s as a rounded
 * difference (TwoSum error-free transform), <n, v> error-free, |h|^2 */
static void source_terms(float ox, float oy, float oz, const f4* s4, const f4* n4, float* hx, float* hy, float* hz,
                         float* nv, float* d2) {
    *hx = ox - s4->x;
    *hy = oy - s4->y;
    *hz = oz - s4->z;
    const float qx = *hx - ox, qy = *hy - oy, qz = *hz - oz;
    const float lx = (ox - (*hx - qx)) + (-s4->x - qx);
    const float ly = (oy - (*hy - qy)) + (-s4->y - qy);
    const float lz = (oz - (*hz - qz)) + (-s4->z - qz);
    const float p = n4->x * *hx;
    float err = fmaf(n4->x, *hx, -p);
    err = fmaf(n4->x, lx, err);
    float acc = p;
    {
        const float p2 = n4->y * *hy;
        const float e2 = fmaf(n4->y, *hy, -p2);
        const float s = acc + p2;
        const float z = s - acc;
        const float q = (acc - (s - z)) + (p2 - z);
        acc = s;
        err = err + (q + e2);
        err = fmaf(n4->y, ly, err);
    }
    {
        const float p3 = n4->z * *hz;
        const float e3 = fmaf(n4->z, *hz, -p3);
        const float s = acc + p3;
        const float z = s - acc;
        const float q = (acc - (s - z)) + (p3 - z);
        acc = s;
        err = err + (q + e3);
        err = fmaf(n4->z, lz, err);
    }
    *nv = acc + err;
    *d2 = fmaf(*hx, *hx, fmaf(*hy, *hy, *hz * *hz));
}

/* per-lane wedge state */
typedef struct {
    float oxn, oxf, oyn, oyf;   /* -(c.x +- delta) / g.x and the same in y: the slab FMAs' addends */
    float igx, igy, zl, zh, sl, sh, lend, ig2, mz;
    int nx_hi, ny_hi;   /* near planes are the upper bounds (direction < 0) */
} wedge_t;

static void wedge_z(wedge_t* w, uint32_t want, float cz, const lamp_t* L, float sz, float delta) {
    float zlo = 3.0e38f, zhi = -3.0e38f;
    for (uint32_t b = want; b; b &= b - 1) {
        const float oz = cz + L->oz[__builtin_ctz(b)];
        zlo = fminf(zlo, oz);
        zhi = fmaxf(zhi, oz);
    }
    w->zl = zlo - delta;
    w->zh = zhi + delta;
    w->sl = sz - zlo;
    w->sh = sz - zhi;
}

static uint32_t lamp_interval(const wedge_t* w, uint32_t want, const f4* a, const f4* b, const f4* c, float cx,
                              float cy, float cz, float sz, float gx, float gy, const lamp_t* L) {
    const float la = fmaf(a->x - cx, gx, (a->y - cy) * gy) * w->ig2;
    const float lb = fmaf(b->x - cx, gx, (b->y - cy) * gy) * w->ig2;
    const float lc = fmaf(c->x - cx, gx, (c->y - cy) * gy) * w->ig2;
    const float lmax = fmax3(la, lb, lc);
    if (!(lmax < 0.9990234375f)) return want;
    const float za = fmaf(a->z - sz, 1.0f / (1.f - la), sz);
    const float zb = fmaf(b->z - sz, 1.0f / (1.f - lb), sz);
    const float zc = fmaf(c->z - sz, 1.0f / (1.f - lc), sz);
    const float m = w->mz * (1.0f / (1.f - lmax));
    const float z0 = fmin3(za, zb, zc) - m, z1 = fmax3(za, zb, zc) + m;
    if (L->wuniform) {
        const float t0 = fminf(fmaxf((z0 - cz - L->wz0) * L->wrdz, -4.f), 40.f);
        const float t1 = fminf(fmaxf((z1 - cz - L->wz0) * L->wrdz, -4.f), 40.f);
        int qlo = (int)ceilf(t0 - 0.03125f), qhi = (int)floorf(t1 + 0.03125f);
        if (qlo < 0) qlo = 0;
        if (qhi > L->K - 1) qhi = L->K - 1;
        if (qhi < qlo) return 0u;
        return want & ((2u << qhi) - 1u) & ~((1u << qlo) - 1u);
    }
    uint32_t in = 0;
    for (uint32_t bits = want; bits; bits &= bits - 1) {
        const int q = __builtin_ctz(bits);
        const float oz = cz + L->oz[q];
        if (oz >= z0 && oz <= z1) in |= 1u << q;
    }
    return in;
}

/* does the lane's wedge meet child boxes (c, c+1) of node nd (pair p = 0, 1) */
static void wedge_pair_hits(const wedge_t* w, const node4_t* nd, int p, int* h0, int* h1) {
    const float* X = nd->q[3 * p], *Y = nd->q[3 * p + 1], *Z = nd->q[3 * p + 2];
    float nx0, nx1, fx0, fx1, ny0, ny1, fy0, fy1;
    if (w->nx_hi) { nx0 = X[2]; nx1 = X[3]; fx0 = X[0]; fx1 = X[1]; }
    else { nx0 = X[0]; nx1 = X[1]; fx0 = X[2]; fx1 = X[3]; }
    if (w->ny_hi) { ny0 = Y[2]; ny1 = Y[3]; fy0 = Y[0]; fy1 = Y[1]; }
    else { ny0 = Y[0]; ny1 = Y[1]; fy0 = Y[2]; fy1 = Y[3]; }
    const float lnx0 = fmaf(nx0, w->igx, w->oxn), lnx1 = fmaf(nx1, w->igx, w->oxn);
    const float lfx0 = fmaf(fx0, w->igx, w->oxf), lfx1 = fmaf(fx1, w->igx, w->oxf);
    const float lny0 = fmaf(ny0, w->igy, w->oyn), lny1 = fmaf(ny1, w->igy, w->oyn);
    const float lfy0 = fmaf(fy0, w->igy, w->oyf), lfy1 = fmaf(fy1, w->igy, w->oyf);
    const float a0 = fmax3(lnx0, lny0, 0.f), a1 = fmax3(lnx1, lny1, 0.f);
    const float b0 = fmin3(lfx0, lfy0, w->lend), b1 = fmin3(lfx1, lfy1, w->lend);
    const float la0 = fmaf(a0, w->sl, w->zl), lb0 = fmaf(b0, w->sl, w->zl);
    const float la1 = fmaf(a1, w->sl, w->zl), lb1 = fmaf(b1, w->sl, w->zl);
    const float ha0 = fmaf(a0, w->sh, w->zh), hb0 = fmaf(b0, w->sh, w->zh);
    const float ha1 = fmaf(a1, w->sh, w->zh), hb1 = fmaf(b1, w->sh, w->zh);
    *h0 = a0 <= b0 && Z[2] >= fminf(la0, lb0) && Z[0] <= fmaxf(ha0, hb0);
    *h1 = a1 <= b1 && Z[3] >= fminf(la1, lb1) && Z[1] <= fmaxf(ha1, hb1);
}

static int lane_beside(const f4* ta, const f4* tb, const f4* tc, float cx, float cy, float gx, float gy, float mh) {
    const float qa = fmaf(ta->x - cx, -gy, (ta->y - cy) * gx);
    const float qb = fmaf(tb->x - cx, -gy, (tb->y - cy) * gx);
    const float qc = fmaf(tc->x - cx, -gy, (tc->y - cy) * gx);
    return (qa > mh && qb > mh && qc > mh) || (qa < -mh && qb < -mh && qc < -mh);
}

typedef struct {
    int valid;
    f4 s, n;
    int32_t ex0, ex1;
    int cache;
    /* per candidate */
    uint32_t want, facing;
    float lend, dmax, gx, gy, mh;
    shear_t sh[MAXK];
    wedge_t w;
} lane_t;

#define QCAP 256
#define QBATCH 32
#ifndef QFLUSH
#define QFLUSH 24   /* the kernels' kLeafFlush */
#endif

/* one queued leaf test for lane P with its sources `snap`: the sources found
 * occluded */
static uint32_t leaf_item(const scene_t* S, const lamp_t* L, const lane_t* P, int leaf, float cx, float cy, float cz,
                          uint32_t snap, uint64_t* C) {
    const f4* t = S->tri + 3 * (size_t)leaf;
    int32_t id;
    memcpy(&id, &t[0].w, 4);
    C[C_LEAF_LOADS]++;
    C[C_PLANE_TESTS]++;
    uint32_t occl = 0;
    if (id != P->ex0 && id != P->ex1 && !lane_beside(&t[0], &t[1], &t[2], cx, cy, P->gx, P->gy, P->mh)) {
        const uint32_t test = snap & lamp_interval(&P->w, snap, &t[0], &t[1], &t[2], cx, cy, cz, P->s.z, P->gx,
                                                   P->gy, L);
        for (uint32_t bits = test; bits; bits &= bits - 1) {
            const int q = __builtin_ctz(bits);
            C[C_TRI_TESTS]++;
            if (seg_tri(cx, cy, cz + L->oz[q], &P->sh[q], &t[0], &t[1], &t[2])) occl |= 1u << q;
        }
    }
    return occl;
}

/* one batch of n <= 32 queued items from the ring position head */
static void leaf_batch(const scene_t* S, const lamp_t* L, lane_t* ln, const int* qlane, const int* qleaf, int head,
                       int n, float cx, float cy, float cz, uint64_t* C) {
    uint32_t snap[32], occ[32];
    int hit[32];
    for (int l = 0; l < 32; ++l) {
        snap[l] = ln[l].want;
        occ[l] = 0;
        hit[l] = -1;
    }
    int nl = 0, uniq = 0;
    int seen_leaf[QBATCH];
    for (int k = 0; k < n; ++k) {
        const int slot = (head + k) & (QCAP - 1), own = qlane[slot], leaf = qleaf[slot];
        if (!snap[own]) continue;   /* the lane has stopped: the item is skipped */
        int seen = 0;
        for (int b = 0; b < nl && !seen; ++b) seen = seen_leaf[b] == leaf;
        seen_leaf[nl++] = leaf;
        uniq += !seen;
        const uint32_t o = leaf_item(S, L, &ln[own], leaf, cx, cy, cz, snap[own], C);
        if (o) {
            occ[own] |= o;
            if (leaf > hit[own]) hit[own] = leaf;
        }
    }
    for (int l = 0; l < 32; ++l) {
        lane_t* P = &ln[l];
        const uint32_t nw = P->want & ~occ[l];
        if (nw != P->want) {
            P->want = nw;
            P->cache = hit[l];
            if (P->want) wedge_z(&P->w, P->want, cz, L, P->s.z, S->cut_eps);
        }
    }
    C[C_LEAF_STEPS]++;
    C[C_LEAF_STEP_LANES] += (uint64_t)nl;
    C[C_LEAF_STEP_UNIQUE] += (uint64_t)uniq;
}

/* one candidate (cx, cy, cz) for the 32 lanes of a task */
static void replay_candidate(const scene_t* S, const lamp_t* L, float cx, float cy, float cz, lane_t* ln,
                             uint64_t* C) {
    const float delta = S->cut_eps;
    for (int l = 0; l < 32; ++l) {
        lane_t* P = &ln[l];
        P->want = 0;
        P->facing = 0;
        P->lend = 0.f;
        P->dmax = 0.f;
        P->gx = 0.f;
        P->gy = 0.f;
        for (int m = 0; m < L->K; ++m) {
            const float ox = cx, oy = cy, oz = cz + L->oz[m];
            float hx, hy, hz, nv, d2;
            source_terms(ox, oy, oz, &P->s, &P->n, &hx, &hy, &hz, &nv, &d2);
            const float d = sqrtf(d2);
            const int fac = P->valid && nv > 0.f && d2 > 0.f;
            P->sh[m] = shear_of(-hx, -hy, -hz);
            const float cut = fmaf(0.99f, P->n.w, -delta);
            const float tend = cut > 0.f ? fmaf(-cut, 1.0f / d, 1.f) : 1.f;
            if (fac) {
                P->facing |= 1u << m;
                if (tend > 0.f) {
                    P->want |= 1u << m;
                    P->lend = fmaxf(P->lend, tend);
                    P->dmax = fmaxf(P->dmax, d);
                }
            }
            P->gx = -hx;
            P->gy = -hy;
        }
        /* wedge_search set-up and the cached occluder */
        const float g2 = fmaf(P->gx, P->gx, P->gy * P->gy);
        const float gn = sqrtf(g2);
        P->mh = delta * gn;
        P->w.ig2 = 1.f / g2;
        P->w.mz = delta * P->dmax / gn;
        if (P->want && P->cache >= 0) {
            const f4* t = S->tri + 3 * (size_t)P->cache;
            C[C_CACHE_LOADS]++;
            const int beside = lane_beside(&t[0], &t[1], &t[2], cx, cy, P->gx, P->gy, P->mh);
            const uint32_t test =
                beside ? 0u : lamp_interval(&P->w, P->want, &t[0], &t[1], &t[2], cx, cy, cz, P->s.z, P->gx, P->gy, L);
            uint32_t occl = 0;
            for (uint32_t bits = test; bits; bits &= bits - 1) {
                const int q = __builtin_ctz(bits);
                if (seg_tri(cx, cy, cz + L->oz[q], &P->sh[q], &t[0], &t[1], &t[2])) occl |= 1u << q;
            }
            P->want &= ~occl;
        }
        C[C_SEARCH_SEGMENTS] += (uint64_t)__builtin_popcount(P->want);
    }
    uint32_t alive = 0;
    for (int l = 0; l < 32; ++l)
        if (ln[l].want) alive |= 1u << l;
    if (!alive || S->nt == 0) return;
    if (S->root < 0) return;   /* a single triangle: no traversal */
    for (int l = 0; l < 32; ++l) {
        lane_t* P = &ln[l];
        wedge_t* w = &P->w;
        const float sgx = signbit(P->gx) ? -delta : delta;
        const float sgy = signbit(P->gy) ? -delta : delta;
        w->igx = safe_rcp(P->gx);
        w->igy = safe_rcp(P->gy);
        w->oxn = -(cx + sgx) * w->igx;
        w->oxf = -(cx - sgx) * w->igx;
        w->oyn = -(cy + sgy) * w->igy;
        w->oyf = -(cy - sgy) * w->igy;
        w->lend = P->lend;
        w->nx_hi = signbit(P->gx) ? 1 : 0;
        w->ny_hi = signbit(P->gy) ? 1 : 0;
        if (P->want) wedge_z(w, P->want, cz, L, P->s.z, delta);
    }
    /* the packet traversal */
    int32_t stack[STACK];
    int qlane[QCAP], qleaf[QCAP], head = 0, tail = 0;
    int top = 0, node = 0;
    uint64_t visits = 0;
    C[C_TRAVERSALS]++;
    while (1) {
        ++visits;
        const node4_t* nd = &S->nodes[node];
        unsigned nib[32], hit = 0;
        C[C_BOX_TESTS] += 4 * (uint64_t)__builtin_popcount(alive);
        C[C_LANE_NODE_VISITS] += (uint64_t)__builtin_popcount(alive);
        for (int l = 0; l < 32; ++l) {
            nib[l] = 0;
            if (!((alive >> l) & 1u)) continue;
            int h0, h1, h2, h3;
            wedge_pair_hits(&ln[l].w, nd, 0, &h0, &h1);
            wedge_pair_hits(&ln[l].w, nd, 1, &h2, &h3);
            nib[l] = (unsigned)h0 | ((unsigned)h1 << 1) | ((unsigned)h2 << 2) | ((unsigned)h3 << 3);
            hit |= nib[l];
        }
        if (hit & (unsigned)nd->m[0]) {
            for (int l = 0; l < 32; ++l)
                for (unsigned b = nib[l] & (unsigned)nd->m[0]; b; b &= b - 1) {
                    qlane[tail & (QCAP - 1)] = l;
                    qleaf[tail & (QCAP - 1)] = ~nd->r[__builtin_ctz(b)];
                    ++tail;
                }
            while (tail - head >= QFLUSH) {
                const int n = tail - head < QBATCH ? tail - head : QBATCH;
                leaf_batch(S, L, ln, qlane, qleaf, head, n, cx, cy, cz, C);
                head += n;
            }
        }
        uint32_t still = 0;
        for (int l = 0; l < 32; ++l)
            if (((alive >> l) & 1u) && ln[l].want) still |= 1u << l;
        alive = still;
        if (!alive) break;
        const unsigned inner = hit & (unsigned)nd->m[1];
        if (inner) {
            const int first = __builtin_ctz(inner);
            const unsigned rest = inner & (inner - 1);
            if (top + 3 > STACK) break;   /* far beyond any tree here */
            stack[top] = nd->r[3]; top += (rest >> 3) & 1u;
            stack[top] = nd->r[2]; top += (rest >> 2) & 1u;
            stack[top] = nd->r[1]; top += (rest >> 1) & 1u;
            node = nd->r[first];
        } else {
            if (top == 0) break;
            node = stack[--top];
        }
    }
    if (tail > head) leaf_batch(S, L, ln, qlane, qleaf, head, tail - head, cx, cy, cz, C);
    C[C_NODE_VISITS] += visits;
}

/*
 * Replay the tasks (chunk ic, patch block jb) listed in `tasks` (ntask pairs)
 * for candidates `cand` (nc x 3, the chunks are cand_per_task consecutive
 * candidates) and add the counters to out[C_NUM] (uint64).  Returns 0, or -1
 * on invalid arguments.
 */
int replay_wedge_tasks(const void* nodes4, const float* tri, const float* patch_s, const float* patch_n,
                       const int32_t* patch_excl, int64_t nt, int64_t np, int32_t root, float diameter,
                       const float* cand, int64_t nc, const float* lamp_oz, int32_t K, int32_t wuniform, float wz0,
                       float wrdz, int32_t cand_per_task, const int64_t* tasks, int64_t ntask, uint64_t* out,
                       int nthreads) {
    if (K < 2 || K > MAXK || cand_per_task < 1 || nt < 1 || np < 0) return -1;
    scene_t S;
    S.nodes = (const node4_t*)nodes4;
    S.tri = (const f4*)tri;
    S.ps = (const f4*)patch_s;
    S.pn = (const f4*)patch_n;
    S.pe = patch_excl;
    S.nt = nt;
    S.np = np;
    S.root = root;
    S.cut_eps = 1e-5f * diameter;
    lamp_t L;
    L.K = K;
    L.wuniform = wuniform;
    L.wz0 = wz0;
    L.wrdz = wrdz;
    for (int m = 0; m < K; ++m) L.oz[m] = lamp_oz[m];
    for (int k = 0; k < C_NUM; ++k) out[k] = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        uint64_t C[C_NUM];
        memset(C, 0, sizeof(C));
#pragma omp for schedule(dynamic, 4)
        for (int64_t k = 0; k < ntask; ++k) {
            const int64_t ic = tasks[2 * k], jb = tasks[2 * k + 1];
            lane_t ln[32];
            for (int l = 0; l < 32; ++l) {
                const int64_t j = jb * 32 + l;
                lane_t* P = &ln[l];
                memset(P, 0, sizeof(*P));
                P->valid = j < np;
                P->ex0 = P->ex1 = -1;
                if (P->valid) {
                    P->s = S.ps[j];
                    P->n = S.pn[j];
                    P->ex0 = S.pe[2 * j];
                    P->ex1 = S.pe[2 * j + 1];
                }
                P->cache = -1;
            }
            C[C_TASKS]++;
            const int64_t i0 = ic * cand_per_task;
            const int64_t i1 = i0 + cand_per_task < nc ? i0 + cand_per_task : nc;
            for (int64_t i = i0; i < i1; ++i) {
                replay_candidate(&S, &L, cand[3 * i], cand[3 * i + 1], cand[3 * i + 2], ln, C);
                for (int l = 0; l < 32; ++l) C[C_PAIRS] += (uint64_t)ln[l].valid;
            }
        }
#pragma omp critical
        for (int q = 0; q < C_NUM; ++q) out[q] += C[q];
    }
    return 0;
}

int replay_num_counters(void) { return C_NUM; }
