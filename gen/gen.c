/*
 * Seeded synthetic inputs for the cluster-relation producer.
 *
 * This module makes meshes, vertex partitions and scalar fields.  It holds no
 * relation arithmetic: both the CPU oracle and the CUDA path read what it
 * writes, and neither shares any other code.
 *
 *  - Freudenthal (Kuhn) subdivision of an n^3 cube grid: every cube is split
 *    into 6 tetrahedra, one per permutation of the three axes.  This stands in
 *    for the paper's tetrahedralised volume datasets (Section 5.1, Table 2).
 *  - Seeded Fisher-Yates permutation of the input vertex ids and optional
 *    uniform jitter of the lattice coordinates.
 *  - kd-tree vertex partition (the clusters, the paper's "segments" of
 *    Section 4.3); fixed leaf cap, or an uneven cap drawn per node.
 *  - Sum-of-Gaussians scalar field.
 *  - Point clouds for the Delaunay generator (gen_delaunay.c).
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood 2014), one stream per use,
 * derived from (seed, stream id).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } rng_t;

static inline uint64_t rng_next(rng_t *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline rng_t rng_make(uint64_t seed, uint64_t stream) {
    rng_t r = {seed * 0xD1B54A32D192ED03ull ^ (stream + 0x8CB92BA72F3D8DD7ull)};
    rng_next(&r);
    return r;
}
/* uniform double in [0,1) with 53 random bits */
static inline double rng_u01(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }
/* uniform integer in [0, m) (multiply-shift, Lemire 2019) */
static inline uint64_t rng_below(rng_t *r, uint64_t m) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * m) >> 64);
}

/* ------------------------------------------------------------------ */
/* Freudenthal grid                                                    */
/* ------------------------------------------------------------------ */

/* The six axis orders, lexicographic.  Tet for order p runs along the path
 * c -> c+e_p0 -> c+e_p0+e_p1 -> c+(1,1,1) through cube corner c. */
static const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

/*
 * n: cubes per axis.  V = (n+1)^3 lattice points, x fastest; T = 6 n^3 tets,
 * cubes x fastest, 6 per cube in kPerm order.
 * permute != 0: input id of lattice point L is perm[L] (Fisher-Yates, stream 1).
 * jitter > 0: coordinates get U(-jitter, +jitter) per axis (stream 2), in
 * lattice order.  Coordinates are in cell units, domain [0, n]^3.
 * xyz: float[V*3] indexed by input id; tv: int32[T*4] of input ids.
 * Returns 0, or -1 if n < 1 or the mesh is too large for int32 ids.
 */
int gen_freudenthal(int32_t n, int32_t permute, double jitter, uint64_t seed, float *xyz, int32_t *tv) {
    if (n < 1) return -1;
    const int64_t m = (int64_t)n + 1;
    const int64_t nv = m * m * m;
    const int64_t nt = 6 * (int64_t)n * n * n;
    if (nv > INT32_MAX || nt * 4 > ((int64_t)1 << 40)) return -1;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * nv);
    if (!perm) return -1;
    for (int64_t i = 0; i < nv; ++i) perm[i] = (int32_t)i;
    if (permute) {
        rng_t r = rng_make(seed, 1);
        for (int64_t i = nv - 1; i > 0; --i) {
            int64_t j = (int64_t)rng_below(&r, (uint64_t)i + 1);
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
    }
    rng_t rj = rng_make(seed, 2);
    for (int64_t k = 0; k < m; ++k)
        for (int64_t j = 0; j < m; ++j)
            for (int64_t i = 0; i < m; ++i) {
                int64_t L = i + m * (j + m * k);
                double p[3] = {(double)i, (double)j, (double)k};
                if (jitter > 0)
                    for (int a = 0; a < 3; ++a) p[a] += (2.0 * rng_u01(&rj) - 1.0) * jitter;
                float *dst = xyz + 3 * (int64_t)perm[L];
                dst[0] = (float)p[0]; dst[1] = (float)p[1]; dst[2] = (float)p[2];
            }
    int64_t t = 0;
    for (int64_t k = 0; k < n; ++k)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i)
                for (int q = 0; q < 6; ++q) {
                    int64_t c[3] = {i, j, k};
                    int32_t *row = tv + 4 * t++;
                    row[0] = perm[c[0] + m * (c[1] + m * c[2])];
                    for (int s = 0; s < 3; ++s) {
                        c[kPerm[q][s]] += 1;
                        row[s + 1] = perm[c[0] + m * (c[1] + m * c[2])];
                    }
                }
    free(perm);
    return 0;
}

/* ------------------------------------------------------------------ */
/* kd-tree partition                                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    const float *xyz;
    int32_t *idx;       /* point ids, reordered so leaves are contiguous in DFS order */
    uint8_t *leaf_start; /* leaf_start[p] = 1 where a leaf begins in idx */
    int32_t cap;         /* fixed cap, or the upper cap of the uneven rule */
    int32_t uneven;
    int32_t min_leaf;    /* uneven rule: nodes below this size always stop */
    int32_t min_cap;     /* uneven rule: lower end of the log-uniform cap draw */
    uint64_t seed;
} kd_ctx;

static inline int kd_less(const float *xyz, int axis, int32_t a, int32_t b) {
    float ca = xyz[3 * (int64_t)a + axis], cb = xyz[3 * (int64_t)b + axis];
    return ca < cb || (ca == cb && a < b);
}

/* Rearrange idx[0..n) so that idx[0..k) hold the k smallest under kd_less
 * (quickselect with median-of-three pivot). */
static void kd_select(const float *xyz, int axis, int32_t *idx, int64_t n, int64_t k) {
    int64_t lo = 0, hi = n - 1;
    while (hi > lo) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t a = idx[lo], b = idx[mid], c = idx[hi], piv;
        if (kd_less(xyz, axis, a, b)) {
            if (kd_less(xyz, axis, b, c)) piv = b; else if (kd_less(xyz, axis, a, c)) piv = c; else piv = a;
        } else {
            if (kd_less(xyz, axis, a, c)) piv = a; else if (kd_less(xyz, axis, b, c)) piv = c; else piv = b;
        }
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (kd_less(xyz, axis, idx[i], piv)) ++i;
            while (kd_less(xyz, axis, piv, idx[j])) --j;
            if (i <= j) { int32_t t = idx[i]; idx[i] = idx[j]; idx[j] = t; ++i; --j; }
        }
        if (k - 1 <= j) hi = j;
        else if (k - 1 >= i) lo = i;
        else break;
    }
}

static int kd_stop(const kd_ctx *c, int64_t n, uint64_t node) {
    if (n <= 1) return 1;
    if (!c->uneven) return n <= c->cap;
    if (n > c->cap) return 0;
    if (n < c->min_leaf) return 1;
    rng_t r = rng_make(c->seed, 0x6B64ull ^ (node << 8));
    double lo = log((double)c->min_cap), hi = log((double)c->cap);
    double cnode = exp(lo + (hi - lo) * rng_u01(&r));
    return (double)n <= cnode;
}

typedef struct { kd_ctx *c; int64_t off, n; uint64_t node; int depth; } kd_job;

static void kd_rec(kd_ctx *c, int64_t off, int64_t n, uint64_t node, int depth);

static void *kd_thread(void *arg) {
    kd_job *j = (kd_job *)arg;
    kd_rec(j->c, j->off, j->n, j->node, j->depth);
    return NULL;
}

static void kd_rec(kd_ctx *c, int64_t off, int64_t n, uint64_t node, int depth) {
    if (kd_stop(c, n, node)) { c->leaf_start[off] = 1; return; }
    int32_t *idx = c->idx + off;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t p = 0; p < n; ++p) {
        const float *q = c->xyz + 3 * (int64_t)idx[p];
        for (int a = 0; a < 3; ++a) { if (q[a] < lo[a]) lo[a] = q[a]; if (q[a] > hi[a]) hi[a] = q[a]; }
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a) if (hi[a] - lo[a] > hi[axis] - lo[axis]) axis = a;
    int64_t m = n / 2;
    kd_select(c->xyz, axis, idx, n, m);
    if (depth < 4 && n > 200000) {
        pthread_t th;
        kd_job j = {c, off, m, 2 * node, depth + 1};
        if (pthread_create(&th, NULL, kd_thread, &j) == 0) {
            kd_rec(c, off + m, n - m, 2 * node + 1, depth + 1);
            pthread_join(th, NULL);
            return;
        }
    }
    kd_rec(c, off, m, 2 * node, depth + 1);
    kd_rec(c, off + m, n - m, 2 * node + 1, depth + 1);
}

/*
 * kd-tree leaves as a vertex partition.  Split the axis of largest bounding-box
 * extent (ties: x before y before z); order points by (coordinate, id); the
 * lower floor(n/2) go left.  Fixed rule: stop at n <= cap.  Uneven rule
 * (uneven != 0): stop if n <= cap and (n < min_leaf or n <= c_node), c_node
 * log-uniform in [min_cap, cap] drawn from (seed, node id), root id 1,
 * children 2i and 2i+1.  Leaves are numbered depth first, left first.
 * seg: int32[nv] leaf id per vertex.  Returns the number of leaves, or -1.
 */
int32_t gen_kdtree(int64_t nv, const float *xyz, int32_t cap, int32_t uneven, int32_t min_leaf,
                   int32_t min_cap, uint64_t seed, int32_t *seg) {
    if (nv < 1 || cap < 1) return -1;
    kd_ctx c = {xyz, NULL, NULL, cap, uneven, min_leaf, min_cap < 1 ? 1 : min_cap, seed};
    c.idx = (int32_t *)malloc(sizeof(int32_t) * nv);
    c.leaf_start = (uint8_t *)calloc((size_t)nv, 1);
    if (!c.idx || !c.leaf_start) { free(c.idx); free(c.leaf_start); return -1; }
    for (int64_t i = 0; i < nv; ++i) c.idx[i] = (int32_t)i;
    kd_rec(&c, 0, nv, 1, 0);
    int32_t leaf = -1;
    for (int64_t p = 0; p < nv; ++p) {
        if (c.leaf_start[p]) ++leaf;
        seg[c.idx[p]] = leaf;
    }
    free(c.idx); free(c.leaf_start);
    return leaf + 1;
}

/* ------------------------------------------------------------------ */
/* Scalar field                                                        */
/* ------------------------------------------------------------------ */

/*
 * f(x) = sum_g a_g exp(-|x - c_g|^2 / (2 s_g^2)), centres uniform in the box
 * [lo, hi], s_g = U[0.05, 0.25] * L with L the largest box extent, amplitudes
 * U[-1, 1].  Evaluated in double, rounded to float.
 */
int gen_field(int64_t nv, const float *xyz, int32_t ngauss, const double *lo, const double *hi, uint64_t seed,
              float *f) {
    if (ngauss < 1 || ngauss > 1024) return -1;
    double cen[1024][3], sig[1024], amp[1024];
    double L = 0;
    for (int a = 0; a < 3; ++a) if (hi[a] - lo[a] > L) L = hi[a] - lo[a];
    rng_t r = rng_make(seed, 3);
    for (int g = 0; g < ngauss; ++g) {
        for (int a = 0; a < 3; ++a) cen[g][a] = lo[a] + (hi[a] - lo[a]) * rng_u01(&r);
        sig[g] = (0.05 + 0.20 * rng_u01(&r)) * L;
        amp[g] = 2.0 * rng_u01(&r) - 1.0;
    }
    for (int64_t v = 0; v < nv; ++v) {
        double s = 0;
        for (int g = 0; g < ngauss; ++g) {
            double d2 = 0;
            for (int a = 0; a < 3; ++a) { double d = (double)xyz[3 * v + a] - cen[g][a]; d2 += d * d; }
            s += amp[g] * exp(-d2 / (2.0 * sig[g] * sig[g]));
        }
        f[v] = (float)s;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Point clouds                                                        */
/* ------------------------------------------------------------------ */

/*
 * n points in [0,1]^3: a fraction frac_mix from a mixture of nmix isotropic
 * Gaussians (sigma U[smin, smax], centres U[0,1]^3, draws outside the unit cube
 * are redrawn), the rest uniform.  Snapped to the integer grid [0, 2^bits) and
 * written as int64 triples; duplicates are not removed here.
 */
int gen_points(int64_t n, double frac_mix, int32_t nmix, double smin, double smax, int32_t bits, uint64_t seed,
               int64_t *pts) {
    if (nmix < 1 || nmix > 64 || bits < 4 || bits > 30) return -1;
    rng_t r = rng_make(seed, 4);
    double cen[64][3], sig[64];
    for (int g = 0; g < nmix; ++g) {
        for (int a = 0; a < 3; ++a) cen[g][a] = rng_u01(&r);
        sig[g] = smin + (smax - smin) * rng_u01(&r);
    }
    const double scale = (double)((int64_t)1 << bits);
    int64_t nmixed = (int64_t)floor(frac_mix * (double)n + 0.5);
    for (int64_t i = 0; i < n; ++i) {
        double p[3];
        if (i < nmixed) {
            int g = (int)rng_below(&r, (uint64_t)nmix);
            for (int a = 0; a < 3; ++a) {
                double x;
                do {
                    /* Box-Muller */
                    double u1 = rng_u01(&r), u2 = rng_u01(&r);
                    if (u1 < 1e-300) u1 = 1e-300;
                    x = cen[g][a] + sig[g] * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
                } while (x < 0.0 || x >= 1.0);
                p[a] = x;
            }
        } else {
            for (int a = 0; a < 3; ++a) p[a] = rng_u01(&r);
        }
        for (int a = 0; a < 3; ++a) {
            int64_t q = (int64_t)floor(p[a] * scale);
            if (q < 0) q = 0;
            if (q >= (int64_t)1 << bits) q = ((int64_t)1 << bits) - 1;
            pts[3 * i + a] = q;
        }
    }
    return 0;
}

/* Seeded Fisher-Yates permutation of [0, n) (stream 5). */
int gen_permutation(int64_t n, uint64_t seed, int32_t *perm) {
    if (n < 0 || n > INT32_MAX) return -1;
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    rng_t r = rng_make(seed, 5);
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)rng_below(&r, (uint64_t)i + 1);
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    return 0;
}
