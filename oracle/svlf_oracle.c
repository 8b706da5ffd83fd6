/*
 * SVLF CPU oracle, traversal part (FP64). TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the package's smoke() check and bench.py's CPU-baseline leg may
 * load this library. It shares no code with the CUDA path.
 *
 * What it computes (the plain definitions, widened from the float32 inputs):
 *
 *  - Leaves are the occupied finest-level voxels of the sparse octree
 *    (Sec. 4.1, "Scene volume"); voxel (i,j,k) at depth L is the box
 *    [i,i+1] x [j,j+1] x [k,k+1] * 2^-L. A leaf's rank is its index in
 *    ascending Morton order (bit 3b = x_b, 3b+1 = y_b, 3b+2 = z_b).
 *
 *  - Ray/voxel intersection uses the slab test (Sec. 4.2 cites an efficient
 *    ray-AABB algorithm for x1, x2): for every axis the ray parameter at the
 *    plane k*2^-L is t = (k*2^-L - o) / d; t_in = max(0, max over axes of the
 *    entering plane), t_out = min over axes of the leaving plane. A voxel is
 *    hit when t_out - t_in > 0.
 *
 *  - The hit list of a ray is its hit voxels in ascending t_in ("indexed by
 *    the order of their intersection along the ray", Sec. 4.3, Eq. 3), cut
 *    to the first K.
 *
 * Two independent ways to get the hit list are provided, and the tests check
 * that they agree: a brute-force slab test against every leaf, and a
 * finest-grid 3-D DDA (Amanatides & Woo) that walks every voxel the ray
 * passes through and looks each one up in the sorted leaf list.
 *
 * The DDA also flags near-degenerate rays, whose hit list a float32
 * traversal could legitimately get differently (see oracle_trace_dda).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- Morton */
uint64_t oracle_morton(int64_t i, int64_t j, int64_t k, int L) {
    uint64_t c = 0;
    for (int b = 0; b < L; ++b) {
        c |= (uint64_t)((i >> b) & 1) << (3 * b);
        c |= (uint64_t)((j >> b) & 1) << (3 * b + 1);
        c |= (uint64_t)((k >> b) & 1) << (3 * b + 2);
    }
    return c;
}

static void demorton(uint64_t c, int L, int64_t ijk[3]) {
    ijk[0] = ijk[1] = ijk[2] = 0;
    for (int b = 0; b < L; ++b) {
        ijk[0] |= (int64_t)((c >> (3 * b)) & 1) << b;
        ijk[1] |= (int64_t)((c >> (3 * b + 1)) & 1) << b;
        ijk[2] |= (int64_t)((c >> (3 * b + 2)) & 1) << b;
    }
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Sorted, de-duplicated Morton codes of the leaf list. Returns the number of
 * unique leaves, or -1 if a coordinate lies outside [0, 2^L). */
int64_t oracle_leaf_codes(const int32_t *ijk, int64_t n, int L, uint64_t *codes) {
    int64_t side = (int64_t)1 << L;
    for (int64_t q = 0; q < n; ++q) {
        for (int a = 0; a < 3; ++a)
            if (ijk[3 * q + a] < 0 || ijk[3 * q + a] >= side) return -1;
        codes[q] = oracle_morton(ijk[3 * q], ijk[3 * q + 1], ijk[3 * q + 2], L);
    }
    qsort(codes, (size_t)n, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (int64_t q = 0; q < n; ++q)
        if (m == 0 || codes[q] != codes[m - 1]) codes[m++] = codes[q];
    return m;
}

static int64_t find_rank(const uint64_t *codes, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (codes[mid] == key) return mid;
        if (codes[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ---------------------------------------------------------------- slab test */
/* Ray parameter where the ray meets plane index k (position k*h) of axis a. */
static double plane_t(const double o[3], const double d[3], int a, int64_t k, double h) {
    return ((double)k * h - o[a]) / d[a];
}

/* Slab test of the box [lo, hi) in plane indices (per axis) at spacing h.
 * Returns 1 and the interval when t_out - t_in > 0. t_in is clipped at 0. */
static int slab(const double o[3], const double d[3], const int64_t lo[3], const int64_t hi[3],
                double h, double *tin, double *tout) {
    double t0 = 0.0, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < (double)lo[a] * h || o[a] > (double)hi[a] * h) return 0;
            continue;
        }
        double ta = plane_t(o, d, a, lo[a], h), tb = plane_t(o, d, a, hi[a], h);
        double tmn = ta < tb ? ta : tb, tmx = ta < tb ? tb : ta;
        if (tmn > t0) t0 = tmn;
        if (tmx < t1) t1 = tmx;
    }
    *tin = t0;
    *tout = t1;
    return t1 - t0 > 0.0;
}

/* --------------------------------------------------------- brute force */
typedef struct { double tin, tout; int64_t rank; } hitrec;

static int cmp_hit(const void *a, const void *b) {
    const hitrec *x = (const hitrec *)a, *y = (const hitrec *)b;
    if (x->tin != y->tin) return x->tin < y->tin ? -1 : 1;
    if (x->tout != y->tout) return x->tout < y->tout ? -1 : 1;
    return x->rank < y->rank ? -1 : (x->rank > y->rank ? 1 : 0);
}

/* All leaves against every ray; hits sorted by (t_in, t_out, rank), first K
 * kept. hit_rank[r*K + j] = -1 for empty slots. */
void oracle_trace_brute(const uint64_t *codes, int64_t n_leaves, int L, const float *rays,
                        int64_t n_rays, int K, int32_t *hit_rank, double *t_in, double *t_out,
                        int32_t *n_hits) {
    double h = ldexp(1.0, -L);
    int64_t (*ijk)[3] = malloc(sizeof(int64_t[3]) * (size_t)(n_leaves > 0 ? n_leaves : 1));
    for (int64_t q = 0; q < n_leaves; ++q) demorton(codes[q], L, ijk[q]);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < n_rays; ++r) {
        double o[3], d[3];
        for (int a = 0; a < 3; ++a) { o[a] = rays[6 * r + a]; d[a] = rays[6 * r + 3 + a]; }
        int cap = 64, n = 0;
        hitrec *buf = malloc(sizeof(hitrec) * (size_t)cap);
        for (int64_t q = 0; q < n_leaves; ++q) {
            int64_t hi[3] = {ijk[q][0] + 1, ijk[q][1] + 1, ijk[q][2] + 1};
            double a0, a1;
            if (slab(o, d, ijk[q], hi, h, &a0, &a1)) {
                if (n == cap) { cap *= 2; buf = realloc(buf, sizeof(hitrec) * (size_t)cap); }
                buf[n].tin = a0; buf[n].tout = a1; buf[n].rank = q; ++n;
            }
        }
        qsort(buf, (size_t)n, sizeof(hitrec), cmp_hit);
        int m = n < K ? n : K;
        n_hits[r] = m;
        for (int j = 0; j < K; ++j) {
            hit_rank[r * K + j] = j < m ? (int32_t)buf[j].rank : -1;
            t_in[r * K + j] = j < m ? buf[j].tin : 0.0;
            t_out[r * K + j] = j < m ? buf[j].tout : 0.0;
        }
        free(buf);
    }
    free(ijk);
}

/* ----------------------------------------------------------------- DDA */
/* Index of the cell along axis a that the ray occupies just after time t:
 * every plane whose crossing time is <= t counts as crossed. */
static int64_t cell_after(const double o[3], const double d[3], int a, double t, int64_t n,
                          double h) {
    if (d[a] == 0.0) {
        int64_t k = (int64_t)floor(o[a] / h);
        return k < 0 ? 0 : (k > n - 1 ? n - 1 : k);
    }
    int64_t k = (int64_t)floor((o[a] + t * d[a]) / h);
    if (k < 0) k = 0;
    if (k > n - 1) k = n - 1;
    if (d[a] > 0) { /* in cell k while plane k crossed and plane k+1 not */
        while (k > 0 && plane_t(o, d, a, k, h) > t) --k;
        while (k < n - 1 && plane_t(o, d, a, k + 1, h) <= t) ++k;
    } else {        /* moving down: in cell k while plane k+1 crossed and plane k not */
        while (k < n - 1 && plane_t(o, d, a, k + 1, h) > t) ++k;
        while (k > 0 && plane_t(o, d, a, k, h) <= t) --k;
    }
    return k;
}

/* Is the cell c + (sum of steps over the axes in `mask`) * sign(d) a leaf?
 * `sgn` = +1/-1 applies the steps forwards or backwards. */
static int stepped_is_leaf(const uint64_t *codes, int64_t n_leaves, int L, const int64_t c[3],
                           const double d[3], int mask, int sgn) {
    int64_t n = (int64_t)1 << L, x[3];
    for (int a = 0; a < 3; ++a) {
        x[a] = c[a] + (((mask >> a) & 1) ? sgn * (d[a] > 0 ? 1 : -1) : 0);
        if (x[a] < 0 || x[a] >= n) return 0;
    }
    return find_rank(codes, n_leaves, oracle_morton(x[0], x[1], x[2], L)) >= 0;
}

/* Finest-grid DDA (Amanatides & Woo): walk every voxel the ray passes
 * through, in order, and keep the leaves. Also returns, per ray, where the
 * inspection started (root entry; -1 for a ray that misses the unit cube) and
 * stopped (t_out of the K-th hit, else the root exit), the number of voxels
 * walked, and a near-degenerate flag.
 *
 * Near-degenerate: a float32 traversal computes each plane crossing to within
 * a few 1e-7 in t (for t below about 4), so it can only disagree with this
 * walk where two crossings of different axes lie within eps = 1e-6 of each
 * other. At such a cluster of crossings, the voxels a different ordering would
 * pass through are the current voxel stepped along any proper, non-empty
 * subset of the clustered axes. The ray is flagged when one of those voxels
 * is a leaf (the hit list could then differ), when its first voxel is shorter
 * than eps, when an axis crossed within eps before the root entry could be
 * counted either way, or when the root test itself is within eps of flipping.
 */
void oracle_trace_dda(const uint64_t *codes, int64_t n_leaves, int L, const float *rays,
                      int64_t n_rays, int K, int32_t *hit_rank, double *t_in, double *t_out,
                      int32_t *n_hits, double *t_start, double *t_end, int64_t *walked,
                      int32_t *degenerate) {
    const double eps = 1e-6;
    double h = ldexp(1.0, -L);
    int64_t n = (int64_t)1 << L;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n_rays; ++r) {
        double o[3], d[3];
        for (int a = 0; a < 3; ++a) { o[a] = rays[6 * r + a]; d[a] = rays[6 * r + 3 + a]; }
        for (int j = 0; j < K; ++j) { hit_rank[r * K + j] = -1; t_in[r * K + j] = 0; t_out[r * K + j] = 0; }
        n_hits[r] = 0;
        walked[r] = 0;
        t_start[r] = -1.0;
        t_end[r] = -1.0;
        degenerate[r] = 0;
        int64_t lo0[3] = {0, 0, 0}, hi0[3] = {n, n, n};
        double te, tx;
        int inside = slab(o, d, lo0, hi0, h, &te, &tx);
        if (fabs(tx - te) < eps) degenerate[r] = 1;
        if (!inside) continue;
        t_start[r] = te;
        int64_t c[3];
        for (int a = 0; a < 3; ++a) c[a] = cell_after(o, d, a, te, n, h);
        /* axes whose last crossing before the entry is within eps of it */
        {
            int entry = -1, late = 0;
            double tp[3];
            for (int a = 0; a < 3; ++a) {
                tp[a] = d[a] > 0 ? plane_t(o, d, a, c[a], h)
                      : d[a] < 0 ? plane_t(o, d, a, c[a] + 1, h) : -INFINITY;
                if (entry < 0 || tp[a] > tp[entry]) entry = a;
            }
            for (int a = 0; a < 3; ++a)
                if (a != entry && d[a] != 0.0 && te - tp[a] < eps) late |= 1 << a;
            for (int sub = 1; sub < 8; ++sub)
                if ((sub & late) == sub && stepped_is_leaf(codes, n_leaves, L, c, d, sub, -1))
                    degenerate[r] = 1;
        }
        double t = te;
        int m = 0;
        int64_t guard = 3 * n + 8;
        int first = 1;
        while (guard-- > 0) {
            double nx[3], tn = INFINITY;
            for (int a = 0; a < 3; ++a) {
                nx[a] = d[a] > 0 ? plane_t(o, d, a, c[a] + 1, h)
                      : d[a] < 0 ? plane_t(o, d, a, c[a], h) : INFINITY;
                if (nx[a] < tn) tn = nx[a];
            }
            if (first && tn - t < eps && find_rank(codes, n_leaves, oracle_morton(c[0], c[1], c[2], L)) >= 0)
                degenerate[r] = 1;
            first = 0;
            int cluster = 0, nclu = 0;
            for (int a = 0; a < 3; ++a)
                if (nx[a] - tn < eps) { cluster |= 1 << a; ++nclu; }
            if (nclu >= 2)
                for (int sub = 1; sub < 7; ++sub)
                    if ((sub & cluster) == sub && sub != cluster &&
                        stepped_is_leaf(codes, n_leaves, L, c, d, sub, +1))
                        degenerate[r] = 1;
            walked[r]++;
            int64_t rank = find_rank(codes, n_leaves, oracle_morton(c[0], c[1], c[2], L));
            if (rank >= 0) {
                int64_t hi[3] = {c[0] + 1, c[1] + 1, c[2] + 1};
                double a0, a1;
                if (slab(o, d, c, hi, h, &a0, &a1)) {
                    hit_rank[r * K + m] = (int32_t)rank;
                    t_in[r * K + m] = a0;
                    t_out[r * K + m] = a1;
                    ++m;
                    if (m == K) { t = tn; break; }
                }
            }
            int out = 0;
            for (int a = 0; a < 3; ++a) {
                if (nx[a] <= tn) {
                    c[a] += d[a] > 0 ? 1 : -1;
                    if (c[a] < 0 || c[a] >= n) out = 1;
                }
            }
            t = tn;
            if (out) break;
        }
        n_hits[r] = m;
        t_end[r] = t;
    }
}

