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
