/*
 * Seeded synthetic scene voxeliser (input generation only).
 *
 * Produces the occupied finest-level voxels ("leaves") of a sparse octree over
 * the unit cube, for a union of solid spheres and axis-aligned box shells.
 * A voxel is occupied when the union signed distance at its centre is within
 * one voxel width of zero, |SDF(centre)| <= 2^-L. This stands in for the
 * paper's octree built from depth maps, which keeps only voxels that contain
 * a surface (Sec. 4.1, "Scene volume"; 128^3 resolution in Sec. 4.5).
 *
 * This file holds none of the rendering method's arithmetic: it only decides
 * which voxels exist. Both the CUDA path and the CPU oracle receive its output
 * as an input array.
 *
 * Method: top-down subdivision. The union SDF is 1-Lipschitz, so a cell whose
 * centre value exceeds (cell half-diagonal - leaf half-diagonal) + 2^-L in
 * magnitude holds no leaf centre satisfying the rule and is pruned. Each cell
 * carries the list of primitives that can still be the minimum anywhere in
 * it. Children are visited in Morton octant order (bit 0 = x, 1 = y, 2 = z),
 * so leaves come out sorted by Morton code.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n_sph, n_box;
    const double *sph;  /* n_sph x 4: cx, cy, cz, r */
    const double *box;  /* n_box x 6: cx, cy, cz, hx, hy, hz */
    int L;
    int32_t *out;       /* capacity x 3 */
    int64_t cap, n;
    int overflow;
} vox_ctx;

static double prim_sdf(const vox_ctx *c, int p, double x, double y, double z) {
    if (p < c->n_sph) {
        const double *s = c->sph + 4 * p;
        double dx = x - s[0], dy = y - s[1], dz = z - s[2];
        return sqrt(dx * dx + dy * dy + dz * dz) - s[3];
    }
    const double *b = c->box + 6 * (p - c->n_sph);
    double qx = fabs(x - b[0]) - b[3];
    double qy = fabs(y - b[1]) - b[4];
    double qz = fabs(z - b[2]) - b[5];
    double ox = qx > 0 ? qx : 0, oy = qy > 0 ? qy : 0, oz = qz > 0 ? qz : 0;
    double outside = sqrt(ox * ox + oy * oy + oz * oz);
    double m = qx > qy ? qx : qy;
    m = m > qz ? m : qz;
    double inside = m < 0 ? m : 0;
    return fabs(outside + inside); /* shell: unsigned distance to the box surface */
}

static void recurse(vox_ctx *c, int level, int64_t i, int64_t j, int64_t k,
                    const int *prims, int np) {
    double w = ldexp(1.0, -level);
    double x = (i + 0.5) * w, y = (j + 0.5) * w, z = (k + 0.5) * w;
    double hL = ldexp(1.0, -c->L);
    double rho = 0.5 * sqrt(3.0) * (w - hL); /* reach of descendant leaf centres */
    double vals[np > 0 ? np : 1];
    double best = INFINITY;
    for (int q = 0; q < np; ++q) {
        vals[q] = prim_sdf(c, prims[q], x, y, z);
        if (vals[q] < best) best = vals[q];
    }
    if (fabs(best) - rho > hL) return;
    if (level == c->L) {
        if (fabs(best) <= hL) {
            if (c->n < c->cap) {
                c->out[3 * c->n + 0] = (int32_t)i;
                c->out[3 * c->n + 1] = (int32_t)j;
                c->out[3 * c->n + 2] = (int32_t)k;
            } else {
                c->overflow = 1;
            }
            c->n++;
        }
        return;
    }
    int keep[np > 0 ? np : 1];
    int nk = 0;
    for (int q = 0; q < np; ++q)
        if (vals[q] - rho <= best + rho) keep[nk++] = prims[q];
    for (int oct = 0; oct < 8; ++oct)
        recurse(c, level + 1, 2 * i + (oct & 1), 2 * j + ((oct >> 1) & 1),
                2 * k + ((oct >> 2) & 1), keep, nk);
}

/* Returns the number of leaves found (may exceed cap: then only cap are
 * written and the caller retries with a larger buffer). */
int64_t svlf_voxelize_union(const double *sph, int n_sph, const double *box, int n_box,
                            int L, int32_t *out_ijk, int64_t cap) {
    vox_ctx c;
    memset(&c, 0, sizeof(c));
    c.n_sph = n_sph; c.n_box = n_box; c.sph = sph; c.box = box; c.L = L;
    c.out = out_ijk; c.cap = cap;
    int np = n_sph + n_box;
    int *all = (int *)malloc(sizeof(int) * (size_t)(np > 0 ? np : 1));
    for (int q = 0; q < np; ++q) all[q] = q;
    recurse(&c, 0, 0, 0, 0, all, np);
    free(all);
    return c.n;
}

/*
 * Analytic depth targets (input generation only): for each float32 ray, the
 * first t >= 0 at which it meets the surface of any primitive (sphere entry,
 * or its exit when the origin is inside; box-shell slab entry, or exit from
 * inside), in float64. mask = 1 where such a t exists, else depth = 0 and
 * mask = 0. The operations and their order follow the array formulation in
 * inputs/__init__.py (_analytic_depth_numpy), which a test compares this with
 * bit for bit. One OpenMP thread per ray block.
 */
static double np_min(double a, double b) { return (isnan(a) || isnan(b)) ? NAN : (a < b ? a : b); }
static double np_max(double a, double b) { return (isnan(a) || isnan(b)) ? NAN : (a > b ? a : b); }

void svlf_analytic_depth(const float *rays, int64_t n, const double *sph, int n_sph, const double *box,
                         int n_box, float *depth, float *mask) {
#pragma omp parallel for schedule(static, 4096)
    for (int64_t r = 0; r < n; ++r) {
        double o[3], d[3];
        for (int a = 0; a < 3; ++a) {
            o[a] = (double)rays[6 * r + a];
            d[a] = (double)rays[6 * r + 3 + a];
        }
        double best = INFINITY;
        for (int p = 0; p < n_sph; ++p) {
            const double *s = sph + 4 * p;
            double oc[3] = {o[0] - s[0], o[1] - s[1], o[2] - s[2]};
            double A = d[0] * d[0] + d[1] * d[1];
            A = A + d[2] * d[2];
            double B = oc[0] * d[0] + oc[1] * d[1];
            B = B + oc[2] * d[2];
            double C = oc[0] * oc[0] + oc[1] * oc[1];
            C = C + oc[2] * oc[2];
            C = C - s[3] * s[3];
            const double disc = B * B - A * C;
            const int ok = disc >= 0;
            const double sq = sqrt(ok ? disc : 0.0);
            const double t0 = (-B - sq) / A;
            const double t1 = (-B + sq) / A;
            double t = t0 >= 0 ? t0 : t1;
            t = (ok && t >= 0) ? t : INFINITY;
            best = np_min(best, t);
        }
        for (int p = 0; p < n_box; ++p) {
            const double *b = box + 6 * p;
            double tmin = NAN, tmax = NAN;
            for (int a = 0; a < 3; ++a) {
                const double lo = b[a] - b[3 + a], hi = b[a] + b[3 + a];
                const double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
                const double mn = np_min(ta, tb), mx = np_max(ta, tb);
                if (!isnan(mn)) tmin = isnan(tmin) ? mn : (mn > tmin ? mn : tmin);
                if (!isnan(mx)) tmax = isnan(tmax) ? mx : (mx < tmax ? mx : tmax);
            }
            const int hit = tmax >= np_max(tmin, 0.0);
            const double t = tmin >= 0 ? tmin : tmax;
            best = np_min(best, hit ? t : INFINITY);
        }
        const int m = isfinite(best);
        depth[r] = (float)(m ? best : 0.0);
        mask[r] = (float)m;
    }
}
