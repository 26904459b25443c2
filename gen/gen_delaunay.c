/*
 * Delaunay tetrahedralisation by Bowyer-Watson insertion with exact integer
 * predicates (input generation only; no relation arithmetic).
 *
 * Points are integer triples in [0, 2^20).  A super-tetrahedron with
 * vertices within +-2^23 encloses them; orient3d and insphere are evaluated
 * exactly in __int128 (every term of the 4x4 insphere determinant stays
 * below 2^123).  Points are inserted in Morton order; the tet containing the
 * next point is found by a visibility walk from the last created tet; the
 * cavity (tets whose circumsphere strictly contains the point) is found by
 * a search from it and re-triangulated from its boundary faces.  Tets with a
 * super vertex are dropped at the end.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

typedef struct {
    int64_t *p;    /* [(n+4) * 3] coordinates; the last 4 are the super vertices */
    int32_t n;     /* input points */
    int32_t *tv;   /* [cap*4] tet vertices (positive orientation) */
    int32_t *nb;   /* [cap*4] neighbour across the face opposite vertex i, -1 none */
    uint32_t *mark;/* [cap] cavity stamp */
    uint8_t *dead; /* [cap] */
    int32_t cnt, cap;
    int32_t *freel; int32_t nfree, freecap;
} dt_t;

static int64_t det3(int64_t a1, int64_t a2, int64_t a3, int64_t b1, int64_t b2, int64_t b3, int64_t c1, int64_t c2,
                    int64_t c3, i128 *out) {
    i128 r = (i128)a1 * ((i128)b2 * c3 - (i128)b3 * c2) - (i128)a2 * ((i128)b1 * c3 - (i128)b3 * c1) +
             (i128)a3 * ((i128)b1 * c2 - (i128)b2 * c1);
    *out = r;
    return 0;
}

/* sign of det [b-a; c-a; d-a]: > 0 when d lies on the positive side */
static int orient3d(const int64_t *a, const int64_t *b, const int64_t *c, const int64_t *d) {
    i128 r;
    det3(b[0] - a[0], b[1] - a[1], b[2] - a[2], c[0] - a[0], c[1] - a[1], c[2] - a[2], d[0] - a[0], d[1] - a[1],
         d[2] - a[2], &r);
    return (r > 0) - (r < 0);
}

/* > 0 iff e lies strictly inside the circumsphere of the positively
 * oriented tet (a, b, c, d) */
static int insphere(const int64_t *a, const int64_t *b, const int64_t *c, const int64_t *d, const int64_t *e) {
    const int64_t *q[4] = {a, b, c, d};
    int64_t m[4][4];
    for (int i = 0; i < 4; ++i) {
        int64_t x = q[i][0] - e[0], y = q[i][1] - e[1], z = q[i][2] - e[2];
        m[i][0] = x; m[i][1] = y; m[i][2] = z; m[i][3] = x * x + y * y + z * z;
    }
    /* expand along the lifted column */
    i128 det = 0;
    for (int i = 0; i < 4; ++i) {
        int r[3], c = 0;
        for (int j = 0; j < 4; ++j)
            if (j != i) r[c++] = j;
        i128 minor;
        det3(m[r[0]][0], m[r[0]][1], m[r[0]][2], m[r[1]][0], m[r[1]][1], m[r[1]][2], m[r[2]][0], m[r[2]][1],
             m[r[2]][2], &minor);
        i128 term = minor * (i128)m[i][3];
        /* cofactor sign for column 3: (-1)^(i+3) */
        if ((i + 3) & 1) det -= term; else det += term;
    }
    /* for a positively oriented tet, det < 0 means inside with this layout */
    return det < 0 ? 1 : (det > 0 ? -1 : 0);
}

static int grow(dt_t *T) {
    int32_t nc = T->cap * 2;
    int32_t *tv = (int32_t *)realloc(T->tv, sizeof(int32_t) * 4 * (size_t)nc);
    if (!tv) return -1;
    T->tv = tv;
    int32_t *nb = (int32_t *)realloc(T->nb, sizeof(int32_t) * 4 * (size_t)nc);
    if (!nb) return -1;
    T->nb = nb;
    uint32_t *mk = (uint32_t *)realloc(T->mark, sizeof(uint32_t) * (size_t)nc);
    if (!mk) return -1;
    T->mark = mk;
    uint8_t *dd = (uint8_t *)realloc(T->dead, (size_t)nc);
    if (!dd) return -1;
    T->dead = dd;
    memset(T->mark + T->cap, 0, sizeof(uint32_t) * (size_t)(nc - T->cap));
    memset(T->dead + T->cap, 0, (size_t)(nc - T->cap));
    T->cap = nc;
    return 0;
}

static int32_t new_tet(dt_t *T) {
    if (T->nfree > 0) {
        int32_t t = T->freel[--T->nfree];
        T->dead[t] = 0;
        T->mark[t] = 0;
        return t;
    }
    if (T->cnt == T->cap && grow(T) != 0) return -1;
    T->dead[T->cnt] = 0;
    T->mark[T->cnt] = 0;
    return T->cnt++;
}

static int push_free(dt_t *T, int32_t t) {
    if (T->nfree == T->freecap) {
        int32_t nc = T->freecap ? T->freecap * 2 : 1024;
        int32_t *f = (int32_t *)realloc(T->freel, sizeof(int32_t) * (size_t)nc);
        if (!f) return -1;
        T->freel = f;
        T->freecap = nc;
    }
    T->freel[T->nfree++] = t;
    T->dead[t] = 1;
    return 0;
}

static uint64_t spread3(uint64_t x) {
    x &= 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

typedef struct { uint64_t key; int32_t idx; } mkey;
static int cmp_mkey(const void *a, const void *b) {
    const mkey *x = (const mkey *)a, *y = (const mkey *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

int gen_orient3d(const int64_t *a, const int64_t *b, const int64_t *c, const int64_t *d) { return orient3d(a, b, c, d); }
int gen_insphere(const int64_t *a, const int64_t *b, const int64_t *c, const int64_t *d, const int64_t *e) {
    return insphere(a, b, c, d, e);
}

static int32_t *g_result = NULL;
static int64_t g_result_n = 0;

/* face i of tet t: the three vertices other than vertex i, in an order that
 * keeps (face, opposite vertex) positively oriented when the face is read
 * with the new apex replacing vertex i */

int gen_delaunay(int64_t n, const int64_t *pts, void **handle, int64_t *nt_out) {
    (void)handle;
    free(g_result);
    g_result = NULL;
    g_result_n = 0;
    if (n < 4) return -1;
    dt_t T;
    memset(&T, 0, sizeof(T));
    T.n = (int32_t)n;
    T.p = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(n + 4));
    T.cap = (int32_t)(8 * n + 64);
    T.tv = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)T.cap);
    T.nb = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)T.cap);
    T.mark = (uint32_t *)calloc((size_t)T.cap, sizeof(uint32_t));
    T.dead = (uint8_t *)calloc((size_t)T.cap, 1);
    mkey *order = (mkey *)malloc(sizeof(mkey) * (size_t)n);
    int32_t *stack = NULL, *cav = NULL, *bnd = NULL;
    int32_t scap = 0, ccap = 0, bcap = 0;
    if (!T.p || !T.tv || !T.nb || !T.mark || !T.dead || !order) return -2;
    memcpy(T.p, pts, sizeof(int64_t) * 3 * (size_t)n);
    const int64_t S = (int64_t)1 << 21, S2 = (int64_t)1 << 23;
    int64_t sup[4][3] = {{-S, -S, -S}, {S2, -S, -S}, {-S, S2, -S}, {-S, -S, S2}};
    for (int i = 0; i < 4; ++i) memcpy(T.p + 3 * (n + i), sup[i], sizeof(sup[i]));
    /* root tet, positively oriented */
    int32_t r = new_tet(&T);
    int32_t sv[4] = {(int32_t)n, (int32_t)n + 1, (int32_t)n + 2, (int32_t)n + 3};
    if (orient3d(T.p + 3 * sv[0], T.p + 3 * sv[1], T.p + 3 * sv[2], T.p + 3 * sv[3]) < 0) {
        int32_t x = sv[2]; sv[2] = sv[3]; sv[3] = x;
    }
    memcpy(T.tv + 4 * r, sv, sizeof(sv));
    for (int i = 0; i < 4; ++i) T.nb[4 * r + i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        order[i].idx = (int32_t)i;
        order[i].key = spread3((uint64_t)pts[3 * i]) | spread3((uint64_t)pts[3 * i + 1]) << 1 |
                       spread3((uint64_t)pts[3 * i + 2]) << 2;
    }
    qsort(order, (size_t)n, sizeof(mkey), cmp_mkey);
    uint32_t stamp = 0;
    int32_t last = r;
    /* edge table linking the new tets of a cavity; grows with the cavity */
    uint32_t kH = 4096;
    uint64_t *hkey = (uint64_t *)malloc(sizeof(uint64_t) * kH);
    int32_t *hval = (int32_t *)malloc(sizeof(int32_t) * kH);
    uint32_t *hst = (uint32_t *)calloc(kH, sizeof(uint32_t));
    if (!hkey || !hval || !hst) return -2;
    uint32_t hstamp = 0;
    uint64_t walkrng = 0x9E3779B97F4A7C15ull;
    for (int64_t oi = 0; oi < n; ++oi) {
        const int32_t pi = order[oi].idx;
        const int64_t *P = T.p + 3 * (int64_t)pi;
        /* visibility walk */
        int32_t t = last;
        for (int64_t steps = 0;; ++steps) {
            if (steps > 4 * (int64_t)T.cnt + 100) return -3; /* cannot happen for valid meshes */
            int moved = 0;
            walkrng = walkrng * 6364136223846793005ull + 1442695040888963407ull;
            int s0 = (int)(walkrng >> 62);
            for (int k = 0; k < 4; ++k) {
                int i = (s0 + k) & 3;
                int32_t *v = T.tv + 4 * t;
                const int64_t *q[4];
                for (int j = 0; j < 4; ++j) q[j] = T.p + 3 * (int64_t)v[j];
                q[i] = P;
                if (orient3d(q[0], q[1], q[2], q[3]) < 0) {
                    int32_t u = T.nb[4 * t + i];
                    if (u < 0) return -4; /* outside the super tet */
                    t = u;
                    moved = 1;
                    break;
                }
            }
            if (!moved) break;
        }
        /* cavity */
        ++stamp;
        int32_t nc = 0, ns = 0, nbnd = 0;
        if (scap == 0) { scap = 1024; stack = (int32_t *)malloc(sizeof(int32_t) * scap); }
        if (ccap == 0) { ccap = 1024; cav = (int32_t *)malloc(sizeof(int32_t) * ccap); }
        if (bcap == 0) { bcap = 2048; bnd = (int32_t *)malloc(sizeof(int32_t) * 2 * bcap); }
        stack[ns++] = t;
        T.mark[t] = stamp;
        while (ns > 0) {
            int32_t c = stack[--ns];
            if (nc == ccap) { ccap *= 2; cav = (int32_t *)realloc(cav, sizeof(int32_t) * ccap); }
            cav[nc++] = c;
            for (int i = 0; i < 4; ++i) {
                int32_t u = T.nb[4 * c + i];
                int inside = 0;
                if (u >= 0 && T.mark[u] != stamp) {
                    const int32_t *w = T.tv + 4 * u;
                    inside = insphere(T.p + 3 * (int64_t)w[0], T.p + 3 * (int64_t)w[1], T.p + 3 * (int64_t)w[2],
                                      T.p + 3 * (int64_t)w[3], P) > 0;
                    if (inside) {
                        T.mark[u] = stamp;
                        if (ns == scap) { scap *= 2; stack = (int32_t *)realloc(stack, sizeof(int32_t) * scap); }
                        stack[ns++] = u;
                    }
                }
                if (u < 0 || (T.mark[u] != stamp)) {
                    if (nbnd == bcap) { bcap *= 2; bnd = (int32_t *)realloc(bnd, sizeof(int32_t) * 2 * bcap); }
                    bnd[2 * nbnd] = c;
                    bnd[2 * nbnd + 1] = i;
                    ++nbnd;
                }
            }
        }
        /* a face may have been recorded as boundary before its neighbour
         * joined the cavity: keep only faces whose neighbour is outside */
        int32_t nb2 = 0;
        for (int32_t b = 0; b < nbnd; ++b) {
            int32_t c = bnd[2 * b], i = bnd[2 * b + 1];
            int32_t u = T.nb[4 * c + i];
            if (u >= 0 && T.mark[u] == stamp) continue;
            bnd[2 * nb2] = c;
            bnd[2 * nb2 + 1] = i;
            ++nb2;
        }
        nbnd = nb2;
        /* new tets: each boundary face with the point replacing the cavity
         * tet's opposite vertex */
        if ((uint32_t)nbnd * 3u > kH / 2u) {
            /* at most 3 edges per new tet: keep the load at or below one half */
            while ((uint32_t)nbnd * 3u > kH / 2u) kH *= 2u;
            free(hkey);
            free(hval);
            free(hst);
            hkey = (uint64_t *)malloc(sizeof(uint64_t) * kH);
            hval = (int32_t *)malloc(sizeof(int32_t) * kH);
            hst = (uint32_t *)calloc(kH, sizeof(uint32_t));
            if (!hkey || !hval || !hst) return -2;
            hstamp = 0;
        }
        int32_t *nt = (int32_t *)malloc(sizeof(int32_t) * (size_t)nbnd);
        for (int32_t b = 0; b < nbnd; ++b) {
            int32_t c = bnd[2 * b], i = bnd[2 * b + 1];
            int32_t x = new_tet(&T);
            if (x < 0) return -2;
            /* c may have been reallocated by grow(): index-based, fine */
            for (int j = 0; j < 4; ++j) T.tv[4 * x + j] = T.tv[4 * c + j];
            T.tv[4 * x + i] = pi;
            for (int j = 0; j < 4; ++j) T.nb[4 * x + j] = -2;
            int32_t u = T.nb[4 * c + i];
            T.nb[4 * x + i] = u;
            if (u >= 0) {
                for (int j = 0; j < 4; ++j)
                    if (T.nb[4 * u + j] == c) T.nb[4 * u + j] = x;
            }
            nt[b] = x;
        }
        /* link new tets across the faces that contain the point: two new
         * tets share such a face iff they share its other two vertices */
        ++hstamp;
        for (int32_t b = 0; b < nbnd; ++b) {
            const int32_t x = nt[b], ip = bnd[2 * b + 1];
            if (orient3d(T.p + 3 * (int64_t)T.tv[4 * x], T.p + 3 * (int64_t)T.tv[4 * x + 1],
                         T.p + 3 * (int64_t)T.tv[4 * x + 2], T.p + 3 * (int64_t)T.tv[4 * x + 3]) <= 0)
                return -5; /* degenerate (flat) tet: points not in general position */
            for (int j = 0; j < 4; ++j) {
                if (j == ip) continue;
                int32_t e[2], c2 = 0;
                for (int q = 0; q < 4; ++q)
                    if (q != j && q != ip) e[c2++] = T.tv[4 * x + q];
                const uint64_t key = e[0] < e[1] ? ((uint64_t)(uint32_t)e[0] << 32 | (uint32_t)e[1])
                                                 : ((uint64_t)(uint32_t)e[1] << 32 | (uint32_t)e[0]);
                uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 32) & (kH - 1u);
                for (;;) {
                    if (hst[h] != hstamp) {
                        hst[h] = hstamp;
                        hkey[h] = key;
                        hval[h] = x * 4 + j;
                        break;
                    }
                    if (hkey[h] == key) {
                        const int32_t y = hval[h] >> 2, jy = hval[h] & 3;
                        T.nb[4 * x + j] = y;
                        T.nb[4 * y + jy] = x;
                        break;
                    }
                    h = (h + 1u) & (kH - 1u);
                }
            }
        }
        for (int32_t c = 0; c < nc; ++c) push_free(&T, cav[c]);
        last = nbnd > 0 ? nt[0] : last;
        free(nt);
    }
    /* collect tets without super vertices */
    int64_t cnt = 0;
    for (int32_t t = 0; t < T.cnt; ++t)
        if (!T.dead[t]) {
            int ok = 1;
            for (int j = 0; j < 4; ++j) ok &= T.tv[4 * t + j] < (int32_t)n;
            cnt += ok;
        }
    g_result = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(cnt ? cnt : 1));
    int64_t w = 0;
    for (int32_t t = 0; t < T.cnt; ++t)
        if (!T.dead[t]) {
            int ok = 1;
            for (int j = 0; j < 4; ++j) ok &= T.tv[4 * t + j] < (int32_t)n;
            if (ok) memcpy(g_result + 4 * w++, T.tv + 4 * t, 16);
        }
    g_result_n = cnt;
    *nt_out = cnt;
    free(T.p); free(T.tv); free(T.nb); free(T.mark); free(T.dead); free(T.freel);
    free(order); free(stack); free(cav); free(bnd);
    free(hkey); free(hval); free(hst);
    return 0;
}

int gen_delaunay_fetch(int32_t *tv) {
    if (!g_result) return -1;
    memcpy(tv, g_result, sizeof(int32_t) * 4 * (size_t)g_result_n);
    free(g_result);
    g_result = NULL;
    return 0;
}
