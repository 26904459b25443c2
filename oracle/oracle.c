/*
 * CPU ORACLE for the cluster-relation producer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code with the CUDA path and nothing in the product links it.
 *
 * It computes, plainly and slowly, what the producer must return: the input
 * checks and the canonical numbering of vertices and tetrahedra (Section 4.3,
 * "Input data" and "Initialization", with the internal/external rule), the
 * per-cluster working sets (internal tets, the external tet list T_ex of
 * Section 4.3, and the face halo TT needs), and the four relations of Table 1
 * that the producer builds (Section 2.2):
 *
 *   VT(v) = { t : v in t }                               (coboundary)
 *   VV(v) = { w != v : v and w lie on a common tet }     (adjacency; the two
 *           vertices share an edge, Section 2.2)
 *   ET(u,w) = { t : u in t and w in t },  u < w          (coboundary)
 *   TT(t) = { t' != t : |t intersect t'| = 3 }           (adjacency: the two
 *           tets share a triangle, Section 2.2)
 *
 * every list ascending.  Readings where the paper is silent:
 *  - canonical vertex ids: vertices stably sorted by (segment, input id), so
 *    every segment owns a contiguous id interval, as the interval arrays I_V of
 *    Section 4.3 presuppose;
 *  - a tet is internal to the segment of its lowest canonical vertex
 *    (Section 4.3), i.e. the smallest segment id among its vertices;
 *  - canonical tet ids: tets stably sorted by (owning segment, input index);
 *  - rows are sets, stored ascending (the paper's kernel fills them in no
 *    fixed order, Algorithm 2);
 *  - edges owned by a segment are those whose lower endpoint it owns, listed
 *    in (u, w) order; TT rows exist for the tets a segment owns.
 *
 * Two independent formulations are provided: the global one (all vertices and
 * tets at once) and a per-cluster one that rescans the whole mesh for one
 * cluster.  The tests check that they agree.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2 };

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

typedef struct { int32_t key, idx; } pair32;
static int cmp_pair32(const void *a, const void *b) {
    const pair32 *x = (const pair32 *)a, *y = (const pair32 *)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->idx > y->idx) - (x->idx < y->idx);
}

typedef struct { int32_t v[4]; } quad32;
static int cmp_quad32(const void *a, const void *b) {
    const quad32 *x = (const quad32 *)a, *y = (const quad32 *)b;
    for (int i = 0; i < 4; ++i)
        if (x->v[i] != y->v[i]) return (x->v[i] > y->v[i]) - (x->v[i] < y->v[i]);
    return 0;
}

static void sort4(int32_t *r) { qsort(r, 4, sizeof(int32_t), cmp_i32); }

/* sort ascending and drop repeats; returns the new length */
static int64_t sort_unique(int32_t *a, int64_t n) {
    if (n == 0) return 0;
    qsort(a, (size_t)n, sizeof(int32_t), cmp_i32);
    int64_t m = 1;
    for (int64_t i = 1; i < n; ++i)
        if (a[i] != a[m - 1]) a[m++] = a[i];
    return m;
}

/* number of vertices two sorted 4-rows share */
static int shared_vertices(const int32_t *a, const int32_t *b) {
    int s = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) s += (a[i] == b[j]);
    return s;
}

/* ------------------------------------------------------------------ */
/* Step 1: input checks (Section 4.3, "Input data")                    */
/* ------------------------------------------------------------------ */

/*
 * The input is V (nv vertices), T (nt tets of 4 vertex ids, the TV relation)
 * and S (a segment id per vertex, nclusters segments).  Accepted iff every
 * id is in range, the 4 ids of a tet are distinct, every segment id is in
 * [0, nclusters), and no two tets have the same vertex set.
 */
int oracle_validate(int64_t nv, int64_t nt, const int32_t *tv, const int32_t *seg, int32_t nclusters) {
    if (nv < 1 || nt < 0 || nclusters < 1 || nv > INT32_MAX || nt > INT32_MAX) return OR_EINVAL;
    for (int64_t v = 0; v < nv; ++v)
        if (seg[v] < 0 || seg[v] >= nclusters) return OR_EINVAL;
    quad32 *q = (quad32 *)malloc(sizeof(quad32) * (size_t)(nt ? nt : 1));
    if (!q) return OR_ENOMEM;
    for (int64_t t = 0; t < nt; ++t) {
        for (int i = 0; i < 4; ++i) {
            int32_t x = tv[4 * t + i];
            if (x < 0 || x >= nv) { free(q); return OR_EINVAL; }
            q[t].v[i] = x;
        }
        sort4(q[t].v);
        for (int i = 1; i < 4; ++i)
            if (q[t].v[i] == q[t].v[i - 1]) { free(q); return OR_EINVAL; }
    }
    qsort(q, (size_t)nt, sizeof(quad32), cmp_quad32);
    for (int64_t t = 1; t < nt; ++t)
        if (cmp_quad32(&q[t], &q[t - 1]) == 0) { free(q); return OR_EINVAL; }
    free(q);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Step 2: canonical vertex ids                                        */
/* ------------------------------------------------------------------ */

/*
 * Vertices sorted by (segment, input id).  cid[v] = rank of input vertex v,
 * vperm[c] = input id of canonical vertex c, I_V[k] = first canonical id of
 * segment k (I_V[nclusters] = nv).  Segment k owns [I_V[k], I_V[k+1]).
 */
int oracle_canon_vertices(int64_t nv, const int32_t *seg, int32_t nclusters, int32_t *cid, int32_t *vperm,
                          int64_t *I_V) {
    pair32 *p = (pair32 *)malloc(sizeof(pair32) * (size_t)nv);
    if (!p) return OR_ENOMEM;
    for (int64_t v = 0; v < nv; ++v) { p[v].key = seg[v]; p[v].idx = (int32_t)v; }
    qsort(p, (size_t)nv, sizeof(pair32), cmp_pair32);
    for (int32_t k = 0; k <= nclusters; ++k) I_V[k] = 0;
    for (int64_t c = 0; c < nv; ++c) {
        vperm[c] = p[c].idx;
        cid[p[c].idx] = (int32_t)c;
        I_V[p[c].key + 1] += 1;
    }
    for (int32_t k = 0; k < nclusters; ++k) I_V[k + 1] += I_V[k];
    free(p);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Step 3: canonical tets                                              */
/* ------------------------------------------------------------------ */

/*
 * Each tet is relabelled to canonical vertex ids and its row sorted
 * ascending, a < b < c < d.  Its owner is the segment of a, its lowest
 * vertex (the internal rule of Section 4.3).  Tets are sorted by
 * (owner, input index): rows[4*t..] is the row of canonical tet t,
 * tperm[t] its input index, and segment k owns tets [I_T[k], I_T[k+1]).
 */
int oracle_canon_tets(int64_t nt, const int32_t *tv, const int32_t *cid, const int32_t *vperm,
                      const int32_t *seg, int32_t nclusters, int32_t *rows, int32_t *tperm, int64_t *I_T) {
    pair32 *p = (pair32 *)malloc(sizeof(pair32) * (size_t)(nt ? nt : 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(nt ? nt : 1));
    if (!p || !tmp) { free(p); free(tmp); return OR_ENOMEM; }
    for (int64_t t = 0; t < nt; ++t) {
        int32_t *r = tmp + 4 * t;
        for (int i = 0; i < 4; ++i) r[i] = cid[tv[4 * t + i]];
        sort4(r);
        p[t].key = seg[vperm[r[0]]]; /* segment of the lowest vertex */
        p[t].idx = (int32_t)t;
    }
    qsort(p, (size_t)nt, sizeof(pair32), cmp_pair32);
    for (int32_t k = 0; k <= nclusters; ++k) I_T[k] = 0;
    for (int64_t t = 0; t < nt; ++t) {
        tperm[t] = p[t].idx;
        memcpy(rows + 4 * t, tmp + 4 * (int64_t)p[t].idx, 4 * sizeof(int32_t));
        I_T[p[t].key + 1] += 1;
    }
    for (int32_t k = 0; k < nclusters; ++k) I_T[k + 1] += I_T[k];
    free(p); free(tmp);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Relations, global formulation                                       */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t nv, nt, ne;
    int64_t *vt_off; int32_t *vt_val;   /* [nv+1], [4 nt] */
    int64_t *vv_off; int32_t *vv_val;   /* [nv+1], [2 ne] */
    int64_t *eu_off;                    /* [nv+1]: edges (u, w), u < w, of vertex u */
    int32_t *e_w;                       /* [ne]: upper endpoint w of each edge */
    int64_t *et_off; int32_t *et_val;   /* [ne+1], [6 nt] */
    int64_t *tt_off; int32_t *tt_val;   /* [nt+1], [sum] */
} oracle_rel;

void oracle_rel_free(oracle_rel *r) {
    if (!r) return;
    free(r->vt_off); free(r->vt_val); free(r->vv_off); free(r->vv_val); free(r->eu_off); free(r->e_w);
    free(r->et_off); free(r->et_val); free(r->tt_off); free(r->tt_val);
    memset(r, 0, sizeof(*r));
}

/* VT over the rows listed in `tets` (ascending), for vertices [v0, v1):
 * each tet is appended, in increasing order, to the row of each of its
 * vertices in range, so every row comes out ascending. */
static int vt_rows(const int32_t *rows, const int32_t *tets, int64_t ntets, int64_t v0, int64_t v1,
                   int64_t **off_out, int32_t **val_out) {
    int64_t n = v1 - v0;
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!off) return OR_ENOMEM;
    for (int64_t i = 0; i < ntets; ++i)
        for (int j = 0; j < 4; ++j) {
            int64_t v = rows[4 * (int64_t)tets[i] + j];
            if (v >= v0 && v < v1) off[v - v0 + 1] += 1;
        }
    for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
    int32_t *val = (int32_t *)malloc(sizeof(int32_t) * (size_t)(off[n] ? off[n] : 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    if (!val || !cur) { free(off); free(val); free(cur); return OR_ENOMEM; }
    for (int64_t v = 0; v < n; ++v) cur[v] = off[v];
    for (int64_t i = 0; i < ntets; ++i)
        for (int j = 0; j < 4; ++j) {
            int64_t v = rows[4 * (int64_t)tets[i] + j];
            if (v >= v0 && v < v1) val[cur[v - v0]++] = tets[i];
        }
    free(cur);
    *off_out = off; *val_out = val;
    return OR_OK;
}

/* VV(v) for each row of a VT CSR: the other vertices of the tets in VT(v),
 * sorted, repeats removed. */
static int vv_from_vt(const int32_t *rows, int64_t v0, int64_t n, const int64_t *vt_off, const int32_t *vt_val,
                      int64_t **off_out, int32_t **val_out) {
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t cap = 3 * (vt_off[n] - vt_off[0]) + 1;
    int32_t *val = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (!off || !val) { free(off); free(val); return OR_ENOMEM; }
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = v0 + i, start = pos;
        for (int64_t q = vt_off[i]; q < vt_off[i + 1]; ++q)
            for (int j = 0; j < 4; ++j) {
                int32_t w = rows[4 * (int64_t)vt_val[q] + j];
                if (w != v) val[pos++] = w;
            }
        pos = start + sort_unique(val + start, pos - start);
        off[i + 1] = pos;
    }
    *off_out = off; *val_out = val;
    return OR_OK;
}

/* ET for the edges whose lower endpoint u is a row of a VT CSR: the pairs
 * (w, t) with t in VT(u), w in t, w > u, sorted by (w, t) and grouped by w.
 * Every tet containing both u and w is in VT(u), so each group is complete. */
static int et_from_vt(const int32_t *rows, int64_t v0, int64_t n, const int64_t *vt_off, const int32_t *vt_val,
                      int64_t **eu_out, int32_t **w_out, int64_t **eoff_out, int32_t **eval_out, int64_t *ne_out) {
    int64_t npairs = 3 * (vt_off[n] - vt_off[0]) + 1;
    pair32 *pr = (pair32 *)malloc(sizeof(pair32) * (size_t)npairs);
    int64_t *eu = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *ew = (int32_t *)malloc(sizeof(int32_t) * (size_t)npairs);
    int64_t *eoff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npairs + 1));
    int32_t *eval = (int32_t *)malloc(sizeof(int32_t) * (size_t)npairs);
    if (!pr || !eu || !ew || !eoff || !eval) { free(pr); free(eu); free(ew); free(eoff); free(eval); return OR_ENOMEM; }
    int64_t ne = 0, nval = 0;
    eoff[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t u = v0 + i, np = 0;
        for (int64_t q = vt_off[i]; q < vt_off[i + 1]; ++q)
            for (int j = 0; j < 4; ++j) {
                int32_t w = rows[4 * (int64_t)vt_val[q] + j];
                if (w > u) { pr[np].key = w; pr[np].idx = vt_val[q]; ++np; }
            }
        qsort(pr, (size_t)np, sizeof(pair32), cmp_pair32);
        for (int64_t p = 0; p < np; ++p) {
            if (p == 0 || pr[p].key != pr[p - 1].key) {
                if (p > 0) eoff[ne + 1] = nval, ++ne;
                ew[ne] = pr[p].key;
            }
            eval[nval++] = pr[p].idx;
        }
        if (np > 0) eoff[ne + 1] = nval, ++ne;
        eu[i + 1] = ne;
    }
    free(pr);
    *eu_out = eu; *w_out = ew; *eoff_out = eoff; *eval_out = eval; *ne_out = ne;
    return OR_OK;
}

/* TT(t) for the tets listed in `tets`: every t' that shares a vertex with t
 * is in VT(x) for some vertex x of t; keep those sharing exactly 3 vertices.
 * vt_off/vt_val index vertex x at row x - vbase and must cover every vertex
 * of the listed tets. */
static int tt_rows(const int32_t *rows, const int32_t *tets, int64_t ntets, int64_t vbase, const int64_t *vt_off,
                   const int32_t *vt_val, int64_t **off_out, int32_t **val_out) {
    int64_t *off = (int64_t *)calloc((size_t)ntets + 1, sizeof(int64_t));
    int32_t *val = (int32_t *)malloc(sizeof(int32_t) * (size_t)(4 * ntets + 1));
    if (!off || !val) { free(off); free(val); return OR_ENOMEM; }
    int32_t *cand = NULL; int64_t ccap = 0;
    int64_t pos = 0;
    for (int64_t i = 0; i < ntets; ++i) {
        int32_t t = tets[i];
        const int32_t *rt = rows + 4 * (int64_t)t;
        int64_t nc = 0;
        for (int j = 0; j < 4; ++j) {
            int64_t x = rt[j] - vbase;
            int64_t len = vt_off[x + 1] - vt_off[x];
            if (nc + len > ccap) {
                ccap = 2 * (nc + len) + 16;
                int32_t *nb = (int32_t *)realloc(cand, sizeof(int32_t) * (size_t)ccap);
                if (!nb) { free(cand); free(off); free(val); return OR_ENOMEM; }
                cand = nb;
            }
            for (int64_t q = vt_off[x]; q < vt_off[x + 1]; ++q) {
                int32_t u = vt_val[q];
                if (u != t && shared_vertices(rt, rows + 4 * (int64_t)u) == 3) cand[nc++] = u;
            }
        }
        nc = sort_unique(cand, nc);
        if (pos + nc > 4 * ntets) { /* non-manifold input: a face in more than two tets */
            int32_t *nb = (int32_t *)realloc(val, sizeof(int32_t) * (size_t)(pos + nc + 4 * ntets));
            if (!nb) { free(cand); free(off); free(val); return OR_ENOMEM; }
            val = nb;
        }
        memcpy(val + pos, cand, sizeof(int32_t) * (size_t)nc);
        pos += nc;
        off[i + 1] = pos;
    }
    free(cand);
    *off_out = off; *val_out = val;
    return OR_OK;
}

/*
 * All four relations over the whole canonical mesh: VT, VV and ET rows for
 * every canonical vertex (ET: every edge, grouped by its lower endpoint), TT
 * rows for every canonical tet.  rows: int32[4 nt], canonical and sorted.
 */
int oracle_relations(int64_t nv, int64_t nt, const int32_t *rows, oracle_rel *out) {
    memset(out, 0, sizeof(*out));
    out->nv = nv; out->nt = nt;
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    if (!all) return OR_ENOMEM;
    for (int64_t t = 0; t < nt; ++t) all[t] = (int32_t)t;
    int rc = vt_rows(rows, all, nt, 0, nv, &out->vt_off, &out->vt_val);
    if (rc == OR_OK) rc = vv_from_vt(rows, 0, nv, out->vt_off, out->vt_val, &out->vv_off, &out->vv_val);
    if (rc == OR_OK)
        rc = et_from_vt(rows, 0, nv, out->vt_off, out->vt_val, &out->eu_off, &out->e_w, &out->et_off, &out->et_val,
                        &out->ne);
    if (rc == OR_OK) rc = tt_rows(rows, all, nt, 0, out->vt_off, out->vt_val, &out->tt_off, &out->tt_val);
    free(all);
    if (rc != OR_OK) oracle_rel_free(out);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Per-cluster formulation                                             */
/* ------------------------------------------------------------------ */

/*
 * The four relations of one cluster k, found by rescanning the whole mesh:
 * VT/VV/ET rows for its vertices [I_V[k], I_V[k+1]) (row i = vertex
 * I_V[k] + i) and TT rows for the tets it owns [I_T[k], I_T[k+1]).
 * Offsets in `out` start at 0 for the cluster.
 */
int oracle_cluster_relations(int64_t nv, int64_t nt, const int32_t *rows, const int64_t *I_V, const int64_t *I_T,
                             int32_t k, oracle_rel *out) {
    memset(out, 0, sizeof(*out));
    const int64_t v0 = I_V[k], v1 = I_V[k + 1];
    out->nv = v1 - v0; out->nt = I_T[k + 1] - I_T[k];
    /* T_k: every tet with a vertex in the cluster */
    int32_t *tk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    if (!tk) return OR_ENOMEM;
    int64_t ntk = 0;
    for (int64_t t = 0; t < nt; ++t) {
        int in = 0;
        for (int j = 0; j < 4; ++j) in |= (rows[4 * t + j] >= v0 && rows[4 * t + j] < v1);
        if (in) tk[ntk++] = (int32_t)t;
    }
    int rc = vt_rows(rows, tk, ntk, v0, v1, &out->vt_off, &out->vt_val);
    if (rc == OR_OK) rc = vv_from_vt(rows, v0, v1 - v0, out->vt_off, out->vt_val, &out->vv_off, &out->vv_val);
    if (rc == OR_OK)
        rc = et_from_vt(rows, v0, v1 - v0, out->vt_off, out->vt_val, &out->eu_off, &out->e_w, &out->et_off,
                        &out->et_val, &out->ne);
    free(tk);
    if (rc != OR_OK) { oracle_rel_free(out); return rc; }

    /* TT of owned tets: star of every vertex of every owned tet */
    uint8_t *mark = (uint8_t *)calloc((size_t)nv, 1);
    if (!mark) { oracle_rel_free(out); return OR_ENOMEM; }
    int64_t vmin = nv, vmax = -1;
    for (int64_t t = I_T[k]; t < I_T[k + 1]; ++t)
        for (int j = 0; j < 4; ++j) {
            int32_t x = rows[4 * t + j];
            mark[x] = 1;
            if (x < vmin) vmin = x;
            if (x > vmax) vmax = x;
        }
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    int32_t *own = (int32_t *)malloc(sizeof(int32_t) * (size_t)(out->nt ? out->nt : 1));
    if (!cand || !own) { free(mark); free(cand); free(own); oracle_rel_free(out); return OR_ENOMEM; }
    int64_t nc = 0;
    for (int64_t t = 0; t < nt; ++t) {
        int in = 0;
        for (int j = 0; j < 4; ++j) in |= mark[rows[4 * t + j]];
        if (in) cand[nc++] = (int32_t)t;
    }
    for (int64_t i = 0; i < out->nt; ++i) own[i] = (int32_t)(I_T[k] + i);
    int64_t *soff = NULL; int32_t *sval = NULL;
    if (vmax >= vmin) {
        /* stars over [vmin, vmax]; vertices outside the marked set are never read */
        rc = vt_rows(rows, cand, nc, vmin, vmax + 1, &soff, &sval);
        if (rc == OR_OK) rc = tt_rows(rows, own, out->nt, vmin, soff, sval, &out->tt_off, &out->tt_val);
    } else {
        out->tt_off = (int64_t *)calloc(1, sizeof(int64_t));
        out->tt_val = (int32_t *)malloc(sizeof(int32_t));
        rc = (out->tt_off && out->tt_val) ? OR_OK : OR_ENOMEM;
    }
    free(soff); free(sval); free(mark); free(cand); free(own);
    if (rc != OR_OK) oracle_rel_free(out);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Working sets                                                        */
/* ------------------------------------------------------------------ */

/*
 * Working set of cluster k (Section 4.3, "Initialization"): T_ex(k), the
 * tets that touch the cluster (a vertex in [I_V[k], I_V[k+1])) but are not
 * internal to it, and the halo H(k), the tets outside T_k that share a
 * triangle with a tet internal to k.  Both ascending.  Caller provides
 * buffers of nt entries each.
 */
int oracle_working_set(int64_t nv, int64_t nt, const int32_t *rows, const int64_t *I_V, const int64_t *I_T,
                       int32_t k, int32_t *ext, int64_t *n_ext, int32_t *halo, int64_t *n_halo) {
    const int64_t v0 = I_V[k], v1 = I_V[k + 1];
    /* a tet sharing a triangle with an internal tet has >= 3 of their vertices */
    uint8_t *mark = (uint8_t *)calloc((size_t)nv, 1);
    if (!mark) return OR_ENOMEM;
    for (int64_t s = I_T[k]; s < I_T[k + 1]; ++s)
        for (int j = 0; j < 4; ++j) mark[rows[4 * s + j]] = 1;
    int64_t ne = 0, nh = 0;
    for (int64_t t = 0; t < nt; ++t) {
        int in = 0, nmark = 0;
        for (int j = 0; j < 4; ++j) {
            in |= (rows[4 * t + j] >= v0 && rows[4 * t + j] < v1);
            nmark += mark[rows[4 * t + j]];
        }
        int owned = (t >= I_T[k] && t < I_T[k + 1]);
        if (in && !owned) ext[ne++] = (int32_t)t;
        if (!in && nmark >= 3) {
            for (int64_t s = I_T[k]; s < I_T[k + 1]; ++s)
                if (shared_vertices(rows + 4 * t, rows + 4 * s) == 3) { halo[nh++] = (int32_t)t; break; }
        }
    }
    free(mark);
    *n_ext = ne; *n_halo = nh;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Per-cluster localized producer                                      */
/* ------------------------------------------------------------------ */

/*
 * The producer's shape on the CPU (Sections 4.3-4.4): an initialisation
 * gathers every cluster's working set once - the tets with a vertex in it
 * (T_k = internal tets + T_ex, Section 4.3) and the face halo that TT needs
 * (tets outside T_k sharing a triangle with an internal tet) - and then each
 * cluster's VT, VV, ET and TT are built from its working set alone, by the
 * same plain definitions as above applied to the working set with its
 * vertices renumbered compactly (an order-preserving map, so every row keeps
 * its ascending order).  Clusters are independent, so nthreads POSIX threads
 * take them from a shared counter.
 */
#include <pthread.h>
#include <time.h>

typedef struct {
    int64_t nv, nt;
    const int32_t *rows;
    const int64_t *I_V, *I_T;
    int32_t K;
    int64_t *ws_off;   /* [K+1] working set of cluster k: ws_val[ws_off[k], ws_off[k+1]) ascending */
    int32_t *ws_val;
} loc_mesh;

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* order-sensitive digest of the ten arrays of one cluster's relations */
static const uint64_t kDigestP[10] = {1000003ull, 1000033ull, 1000037ull, 1000039ull, 1000081ull,
                                      1000099ull, 1000117ull, 1000121ull, 1000133ull, 1000151ull};
static uint64_t digest64(const int64_t *a, int64_t n, int which) {
    uint64_t d = kDigestP[which] * (uint64_t)(n + 1);
    for (int64_t i = 0; i < n; ++i) d += ((uint64_t)a[i] + 7ull) * (uint64_t)(i + 1) * kDigestP[which];
    return d;
}
static uint64_t digest32(const int32_t *a, int64_t n, int which) {
    uint64_t d = kDigestP[which] * (uint64_t)(n + 1);
    for (int64_t i = 0; i < n; ++i) d += ((uint64_t)(int64_t)a[i] + 7ull) * (uint64_t)(i + 1) * kDigestP[which];
    return d;
}

/* Working sets of all clusters (the initialisation).  T_k from one pass over
 * the tets; the halo from the global vertex stars: the tet across the face
 * (b, c, d) of an internal tet whose b is not in the cluster is the other
 * tet of star(b) holding c and d. */
static int loc_working_sets(loc_mesh *m) {
    const int64_t nv = m->nv, nt = m->nt;
    const int32_t *rows = m->rows;
    const int32_t K = m->K;
    int32_t *vc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv ? nv : 1));
    int64_t *cnt = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
    int64_t *soff = NULL; int32_t *sval = NULL;
    int64_t *hoff = NULL; int32_t *hval = NULL;
    if (!vc || !cnt) { free(vc); free(cnt); return OR_ENOMEM; }
    for (int32_t k = 0; k < K; ++k)
        for (int64_t v = m->I_V[k]; v < m->I_V[k + 1]; ++v) vc[v] = k;
    /* global vertex stars */
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    if (!all) { free(vc); free(cnt); return OR_ENOMEM; }
    for (int64_t t = 0; t < nt; ++t) all[t] = (int32_t)t;
    int rc = vt_rows(rows, all, nt, 0, nv, &soff, &sval);
    free(all);
    if (rc != OR_OK) { free(vc); free(cnt); return rc; }
    /* halo lists: count, then fill (duplicates removed per cluster later) */
    hoff = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
    if (!hoff) { free(vc); free(cnt); free(soff); free(sval); return OR_ENOMEM; }
    for (int pass = 0; pass < 2; ++pass) {
        int64_t *fillp = NULL;
        if (pass == 1) {
            for (int32_t k = 0; k < K; ++k) hoff[k + 1] += hoff[k];
            hval = (int32_t *)malloc(sizeof(int32_t) * (size_t)(hoff[K] ? hoff[K] : 1));
            fillp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K ? K : 1));
            if (!hval || !fillp) { free(fillp); free(vc); free(cnt); free(soff); free(sval); free(hoff); free(hval); return OR_ENOMEM; }
            for (int32_t k = 0; k < K; ++k) fillp[k] = hoff[k];
        }
        for (int32_t k = 0; k < K; ++k)
            for (int64_t t = m->I_T[k]; t < m->I_T[k + 1]; ++t) {
                const int32_t *r = rows + 4 * t;
                if (vc[r[1]] == k) continue; /* face (b, c, d) has an own vertex: inside T_k */
                const int32_t b = r[1];
                for (int64_t q = soff[b]; q < soff[b + 1]; ++q) {
                    const int32_t u = sval[q];
                    if (u == (int32_t)t) continue;
                    const int32_t *ru = rows + 4 * (int64_t)u;
                    int hc = 0, hd = 0, in_k = 0;
                    for (int j = 0; j < 4; ++j) {
                        hc |= ru[j] == r[2];
                        hd |= ru[j] == r[3];
                        in_k |= vc[ru[j]] == k;
                    }
                    if (hc && hd && !in_k) {
                        if (pass == 0) hoff[k + 1]++;
                        else hval[fillp[k]++] = u;
                    }
                }
            }
        free(fillp);
    }
    free(soff); free(sval);
    /* T_k: each tet, once for each distinct cluster among its vertices */
    for (int pass = 0; pass < 2; ++pass) {
        int64_t *fillp = NULL;
        if (pass == 1) {
            m->ws_off = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
            if (!m->ws_off) { free(vc); free(cnt); free(hoff); free(hval); return OR_ENOMEM; }
            for (int32_t k = 0; k < K; ++k) m->ws_off[k + 1] = m->ws_off[k] + cnt[k] + (hoff[k + 1] - hoff[k]);
            m->ws_val = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m->ws_off[K] ? m->ws_off[K] : 1));
            fillp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K ? K : 1));
            if (!m->ws_val || !fillp) { free(fillp); free(vc); free(cnt); free(hoff); free(hval); return OR_ENOMEM; }
            for (int32_t k = 0; k < K; ++k) fillp[k] = m->ws_off[k];
        }
        for (int64_t t = 0; t < nt; ++t) {
            int32_t seen[4];
            int ns = 0;
            for (int j = 0; j < 4; ++j) {
                const int32_t c = vc[rows[4 * t + j]];
                int dup = 0;
                for (int i = 0; i < ns; ++i) dup |= seen[i] == c;
                if (dup) continue;
                seen[ns++] = c;
                if (pass == 0) cnt[c]++;
                else m->ws_val[fillp[c]++] = (int32_t)t;
            }
        }
        if (pass == 1) {
            /* halo after T_k, then the whole working set ascending and unique */
            for (int32_t k = 0; k < K; ++k) {
                for (int64_t q = hoff[k]; q < hoff[k + 1]; ++q) m->ws_val[fillp[k]++] = hval[q];
                const int64_t n = fillp[k] - m->ws_off[k];
                const int64_t u = sort_unique(m->ws_val + m->ws_off[k], n);
                for (int64_t q = m->ws_off[k] + u; q < fillp[k]; ++q) m->ws_val[q] = INT32_MAX;
            }
        }
        free(fillp);
    }
    free(vc); free(cnt); free(hoff); free(hval);
    return OR_OK;
}

static int cmp_i32p(const void *a, const void *b) { return cmp_i32(a, b); }

/* The four relations of cluster k from its working set alone; offsets start
 * at 0 for the cluster (the layout of oracle_cluster_relations). */
static int loc_cluster(const loc_mesh *m, int32_t k, oracle_rel *out) {
    memset(out, 0, sizeof(*out));
    const int32_t *ws = m->ws_val + m->ws_off[k];
    int64_t nws = m->ws_off[k + 1] - m->ws_off[k];
    while (nws > 0 && ws[nws - 1] == INT32_MAX) --nws;
    const int64_t v0 = m->I_V[k], v1 = m->I_V[k + 1];
    const int64_t t0 = m->I_T[k], t1 = m->I_T[k + 1];
    out->nv = v1 - v0; out->nt = t1 - t0;
    /* compact vertex numbering of the working set (order preserving) */
    int32_t *vmap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(4 * nws + 1));
    int32_t *lrows = (int32_t *)malloc(sizeof(int32_t) * (size_t)(4 * nws + 1));
    int32_t *lt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nws + 1));
    int32_t *own = (int32_t *)malloc(sizeof(int32_t) * (size_t)(out->nt + 1));
    if (!vmap || !lrows || !lt || !own) { free(vmap); free(lrows); free(lt); free(own); return OR_ENOMEM; }
    for (int64_t i = 0; i < nws; ++i)
        for (int j = 0; j < 4; ++j) vmap[4 * i + j] = m->rows[4 * (int64_t)ws[i] + j];
    const int64_t nloc = sort_unique(vmap, 4 * nws);
    for (int64_t i = 0; i < 4 * nws; ++i) {
        const int32_t g = m->rows[4 * (int64_t)ws[i / 4] + (i % 4)];
        const int32_t *p = (const int32_t *)bsearch(&g, vmap, (size_t)nloc, sizeof(int32_t), cmp_i32p);
        lrows[i] = (int32_t)(p - vmap);
    }
    int64_t n_own = 0;
    for (int64_t i = 0; i < nws; ++i) {
        lt[i] = (int32_t)i;
        if (ws[i] >= t0 && ws[i] < t1) own[n_own++] = (int32_t)i;
    }
    int32_t lo = 0;
    while (lo < nloc && vmap[lo] < v0) ++lo;
    const int64_t nvo = v1 - v0;
    int rc = OR_OK;
    if (n_own != out->nt || (nvo > 0 && (lo + nvo > nloc || vmap[lo] != v0))) rc = OR_EINVAL;
    int64_t *soff = NULL; int32_t *sval = NULL;
    if (rc == OR_OK) rc = vt_rows(lrows, lt, nws, lo, lo + nvo, &out->vt_off, &out->vt_val);
    if (rc == OR_OK) rc = vv_from_vt(lrows, lo, nvo, out->vt_off, out->vt_val, &out->vv_off, &out->vv_val);
    if (rc == OR_OK)
        rc = et_from_vt(lrows, lo, nvo, out->vt_off, out->vt_val, &out->eu_off, &out->e_w, &out->et_off,
                        &out->et_val, &out->ne);
    /* TT of the internal tets: stars of every working-set vertex */
    if (rc == OR_OK) rc = vt_rows(lrows, lt, nws, 0, nloc, &soff, &sval);
    if (rc == OR_OK) rc = tt_rows(lrows, own, n_own, 0, soff, sval, &out->tt_off, &out->tt_val);
    free(soff); free(sval);
    if (rc == OR_OK) {
        /* back to canonical ids */
        for (int64_t q = 0; q < out->vt_off[nvo]; ++q) out->vt_val[q] = ws[out->vt_val[q]];
        for (int64_t q = 0; q < out->vv_off[nvo]; ++q) out->vv_val[q] = vmap[out->vv_val[q]];
        for (int64_t q = 0; q < out->ne; ++q) out->e_w[q] = vmap[out->e_w[q]];
        for (int64_t q = 0; q < out->et_off[out->ne]; ++q) out->et_val[q] = ws[out->et_val[q]];
        for (int64_t q = 0; q < out->tt_off[n_own]; ++q) out->tt_val[q] = ws[out->tt_val[q]];
    }
    free(vmap); free(lrows); free(lt); free(own);
    if (rc != OR_OK) oracle_rel_free(out);
    return rc;
}

typedef struct {
    const loc_mesh *m;
    int64_t *next;   /* shared cluster counter */
    int64_t *sizes;  /* [K][5] */
    uint64_t *digests;
    int err;
} loc_job;

static void *loc_worker(void *arg) {
    loc_job *j = (loc_job *)arg;
    for (;;) {
        const int64_t k = __atomic_fetch_add(j->next, 1, __ATOMIC_RELAXED);
        if (k >= j->m->K) break;
        oracle_rel r;
        if (loc_cluster(j->m, (int32_t)k, &r) != OR_OK) { j->err = 1; continue; }
        const int64_t nvo = r.nv, nown = r.nt;
        int64_t *s = j->sizes + 5 * k;
        s[0] = r.vt_off[nvo]; s[1] = r.vv_off[nvo]; s[2] = r.ne; s[3] = r.et_off[r.ne]; s[4] = r.tt_off[nown];
        if (j->digests)
            j->digests[k] = digest64(r.vt_off, nvo + 1, 0) + digest32(r.vt_val, s[0], 1) + digest64(r.vv_off, nvo + 1, 2) +
                            digest32(r.vv_val, s[1], 3) + digest64(r.eu_off, nvo + 1, 4) + digest32(r.e_w, s[2], 5) +
                            digest64(r.et_off, s[2] + 1, 6) + digest32(r.et_val, s[3], 7) +
                            digest64(r.tt_off, nown + 1, 8) + digest32(r.tt_val, s[4], 9);
        oracle_rel_free(&r);
    }
    return NULL;
}

/*
 * Build every cluster from its working set with nthreads threads.
 *   sizes    int64[K*5] out: per cluster |VT|, |VV|, #edges, |ET|, |TT|
 *   digests  uint64[K] out (may be NULL): digest of the cluster's ten arrays
 *   seconds  double[2] out: initialisation, then the per-cluster builds
 */
int oracle_localized_build(int64_t nv, int64_t nt, const int32_t *rows, const int64_t *I_V, const int64_t *I_T,
                           int32_t K, int32_t nthreads, int64_t *sizes, uint64_t *digests, double *seconds) {
    loc_mesh m = {nv, nt, rows, I_V, I_T, K, NULL, NULL};
    double t0 = now_s();
    int rc = loc_working_sets(&m);
    double t1 = now_s();
    if (rc != OR_OK) return rc;
    if (nthreads < 1) nthreads = 1;
    int64_t next = 0;
    loc_job *jobs = (loc_job *)calloc((size_t)nthreads, sizeof(loc_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); free(m.ws_off); free(m.ws_val); return OR_ENOMEM; }
    int started = 0;
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = (loc_job){&m, &next, sizes, digests, 0};
        if (i == 0 || pthread_create(&th[i], NULL, loc_worker, &jobs[i]) == 0) started = i + 1;
        else break;
    }
    loc_worker(&jobs[0]);  /* the caller's thread is worker 0 */
    for (int i = 1; i < started; ++i) pthread_join(th[i], NULL);
    double t2 = now_s();
    for (int i = 0; i < started; ++i) rc |= jobs[i].err ? OR_EINVAL : OR_OK;
    free(jobs); free(th); free(m.ws_off); free(m.ws_val);
    if (seconds) { seconds[0] = t1 - t0; seconds[1] = t2 - t1; }
    return rc == OR_OK ? OR_OK : OR_EINVAL;
}

/* One cluster of the localized producer, with its working sets gathered
 * first (for tests: the same code path as oracle_localized_build). */
int oracle_localized_cluster(int64_t nv, int64_t nt, const int32_t *rows, const int64_t *I_V, const int64_t *I_T,
                             int32_t K, int32_t k, oracle_rel *out) {
    loc_mesh m = {nv, nt, rows, I_V, I_T, K, NULL, NULL};
    int rc = loc_working_sets(&m);
    if (rc == OR_OK) rc = loc_cluster(&m, k, out);
    free(m.ws_off); free(m.ws_val);
    return rc;
}
