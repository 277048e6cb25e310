/*
 * Plain, slow, single-threaded FP64 oracle for Parallel Toplesets
 * Propagation (PTP), Romero Calla, Fuentes Perez, Montenegro,
 * "A minimalistic approach for fast computation of geodesic distances on
 * triangular meshes".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load or run this code.  It shares no code,
 * header, table or helper with the CUDA library and must never be reached
 * from the library's product path.
 *
 * What it computes, step by step, in the paper's order:
 *   1. vertex -> incident-triangle lists (the mesh adjacency, Sec. 4.3 uses a
 *      compact half-edge structure; any incidence structure gives the same
 *      triangles);
 *   2. toplesets V_r by breadth-first search from the sources (Sec. 4.1,
 *      Definition of the topleset: V_0 = S, V_r = unvisited neighbours of
 *      V_{r-1});
 *   3. the Jacobi iteration d_k = F(d_{k-1}) over the update band
 *      B = V_{i_{k-1}} u ... u V_{j_k} (Sec. 4.2), with the band bounds of
 *      Eq. (upper_band) and Eq. (lower_band);
 *   4. the per-triangle update step: the planar (linear) local solve of the
 *      Eikonal equation |grad d| = 1 (Sec. 2, Eq. 1) inside one triangle,
 *      kept only when the monotonicity condition Q X^T n < 0 of Sec. 3.2
 *      holds, else the edge (Dijkstra-like) fallback.  No unfolding or
 *      subdivision of obtuse triangles is done (Sec. 3.2, Sec. 5).
 *
 * Readings of points the paper leaves open are listed where they are used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_ERR_ARG (-1)
#define OR_ERR_INDEX (-2)
#define OR_ERR_DEGENERATE_FACE (-3)
#define OR_ERR_NOMEM (-4)

/* A triangle is treated as degenerate (edge fallback only) when
 * det = |e1|^2 |e2|^2 - (e1.e2)^2 <= OR_DEGENERATE * |e1|^2 |e2|^2,
 * i.e. the squared sine of its angle at the updated vertex is below 1e-12. */
#define OR_DEGENERATE 1e-12

static double dot3(const double *u, const double *v) {
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}

/*
 * Update step for vertex x0 of triangle (x0, x1, x2) with known distances
 * d1 at x1 and d2 at x2 (Sec. 3.2, the Kimmel-Sethian planar update).
 *
 * Model: d is linear on the triangle, d(x) = p + g.(x - x0), so with
 * X = [e1 e2], e_i = x_i - x0, t = (d1, d2)^T:  X^T g = t - p 1.  Restricted
 * to the triangle's plane g = X Q (t - p 1) with Q = (X^T X)^{-1}.  The
 * Eikonal equation |g| = 1 becomes the quadratic
 *     (1^T Q 1) p^2 - 2 (1^T Q t) p + (t^T Q t - 1) = 0,
 * whose larger root is the arrival time at x0.  With the wavefront normal
 * n = g, Q X^T n = Q X^T X Q (t - p 1) = Q (t - p 1); the monotonicity
 * condition Q X^T n < 0 (componentwise) says the characteristic reaches x0
 * from inside the triangle.  When it fails, or there is no real root, or the
 * triangle is degenerate, the update falls back to the shortest edge path,
 * min(d1 + |e1|, d2 + |e2|).  With only one finite neighbour distance only
 * that edge is available; with none the result is +infinity.
 *
 * Evaluation.  Exact identities of this quadratic keep FP64 accurate on
 * near-degenerate triangles (squared sine of an angle down to 1e-12), where
 * its coefficients as written cancel: det(X^T X) = |e1 x e2|^2; (i) shift
 * invariance -- the model's
 * data t - d1 1 has the root p - d1, so the quadratic is solved for
 * r = p - d1 with t' = (0, d2 - d1); (ii) the whole equation is multiplied
 * by det = det(X^T X), i.e. Q is replaced by its adjugate
 * M = det Q = [[c, -b], [-b, a]], which has the same roots and, det being
 * positive, the same signs in the monotonicity condition M (t' - r 1) < 0.
 * Without them the rounding error of the coefficients grows like
 * (d / |e|)^2 / sin^2 of the smallest angle times the machine epsilon.
 */
double or_update(const double *x0, const double *x1, const double *x2, double d1, double d2) {
    double e1[3], e2[3];
    for (int i = 0; i < 3; ++i) {
        e1[i] = x1[i] - x0[i];
        e2[i] = x2[i] - x0[i];
    }
    const int f1 = isfinite(d1), f2 = isfinite(d2);
    if (!f1 && !f2) return INFINITY;
    const double a = dot3(e1, e1), b = dot3(e1, e2), c = dot3(e2, e2);
    const double edge1 = f1 ? d1 + sqrt(a) : INFINITY;
    const double edge2 = f2 ? d2 + sqrt(c) : INFINITY;
    const double fallback = edge1 < edge2 ? edge1 : edge2;
    if (!f1 || !f2) return fallback;

    /* det(X^T X) = a c - b^2, computed as |e1 x e2|^2 (Lagrange's identity):
     * the difference a c - b^2 cancels when e1 and e2 are nearly parallel */
    const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double det = dot3(cr, cr);
    if (!(det > OR_DEGENERATE * a * c)) return fallback;

    /* M = det Q = [[c, -b], [-b, a]], data t' = (0, delta) for r = p - d1 */
    const double m11 = c, m12 = -b, m22 = a;
    const double t1 = 0.0, t2 = d2 - d1;
    const double qa = m11 + 2.0 * m12 + m22;                                   /* det 1^T Q 1       */
    const double qb = m11 * t1 + m12 * (t1 + t2) + m22 * t2;                   /* det 1^T Q t'      */
    const double qc = m11 * t1 * t1 + 2.0 * m12 * t1 * t2 + m22 * t2 * t2 - det; /* det (t'^T Q t' - 1) */
    const double disc = qb * qb - qa * qc;
    if (disc < 0.0) return fallback;
    const double r = (qb + sqrt(disc)) / qa;

    /* Q (t - p 1) = M (t' - r 1) / det < 0 componentwise */
    const double l1 = m11 * (t1 - r) + m12 * (t2 - r);
    const double l2 = m12 * (t1 - r) + m22 * (t2 - r);
    if (l1 < 0.0 && l2 < 0.0) return d1 + r;
    return fallback;
}

/*
 * Vertex -> incident triangles.  For vertex v, row[v]..row[v+1]-1 index the
 * triangles (v, a, b) that contain v, given as the other two vertices in the
 * face's cyclic order.  Built by counting then filling in face order.
 * Returns OR_ERR_INDEX for an out-of-range index and OR_ERR_DEGENERATE_FACE
 * for a face that repeats a vertex.
 */
int or_incident(int64_t n, int64_t nf, const int32_t *faces, int64_t *row, int32_t *oa, int32_t *ob) {
    if (n <= 0 || nf < 0 || !faces || !row || !oa || !ob) return OR_ERR_ARG;
    for (int64_t f = 0; f < nf; ++f) {
        const int32_t *t = faces + 3 * f;
        for (int s = 0; s < 3; ++s)
            if (t[s] < 0 || t[s] >= n) return OR_ERR_INDEX;
        if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2]) return OR_ERR_DEGENERATE_FACE;
    }
    for (int64_t v = 0; v <= n; ++v) row[v] = 0;
    for (int64_t f = 0; f < 3 * nf; ++f) row[faces[f] + 1] += 1;
    for (int64_t v = 0; v < n; ++v) row[v + 1] += row[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!fill) return OR_ERR_NOMEM;
    for (int64_t v = 0; v < n; ++v) fill[v] = row[v];
    for (int64_t f = 0; f < nf; ++f) {
        const int32_t *t = faces + 3 * f;
        for (int s = 0; s < 3; ++s) {
            const int32_t v = t[s];
            const int64_t slot = fill[v]++;
            oa[slot] = t[(s + 1) % 3];
            ob[slot] = t[(s + 2) % 3];
        }
    }
    free(fill);
    return OR_OK;
}

/*
 * Toplesets (Sec. 4.1, Definition): level[v] = length of the shortest
 * edge path from v to the source set S in the mesh graph, by a FIFO
 * breadth-first search; V_0 = S.  Vertices not reachable from S get -1.
 * Returns rho, the number of toplesets (1 + the largest level), or a
 * negative error.
 */
int64_t or_toplesets(int64_t n, const int64_t *row, const int32_t *oa, const int32_t *ob,
                     int32_t m, const int32_t *src, int32_t *level) {
    if (n <= 0 || m <= 0 || !row || !oa || !ob || !src || !level) return OR_ERR_ARG;
    for (int32_t s = 0; s < m; ++s)
        if (src[s] < 0 || src[s] >= n) return OR_ERR_INDEX;
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!queue) return OR_ERR_NOMEM;
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    int64_t head = 0, tail = 0;
    for (int32_t s = 0; s < m; ++s) {
        if (level[src[s]] != 0) {
            level[src[s]] = 0;
            queue[tail++] = src[s];
        }
    }
    int64_t rho = 1;
    while (head < tail) {
        const int64_t v = queue[head++];
        for (int64_t c = row[v]; c < row[v + 1]; ++c) {
            const int32_t w2[2] = {oa[c], ob[c]};
            for (int q = 0; q < 2; ++q) {
                const int32_t w = w2[q];
                if (level[w] < 0) {
                    level[w] = level[v] + 1;
                    if (level[w] + 1 > rho) rho = level[w] + 1;
                    queue[tail++] = w;
                }
            }
        }
    }
    free(queue);
    return rho;
}

/* Relative-change test of Eq. (lower_band) for one vertex of V_{i_{k-1}}.
 * Readings: the paper's |d_k - d_{k-1}| / d_{k-1} < eps is undefined for
 * d_{k-1} in {0, inf}; it is evaluated as  delta == 0  or
 * delta < eps * d_{k-1} + eps_abs  (eps_abs = 0 reproduces the paper), and a
 * non-finite d_{k-1} never counts as converged. */
static int converged_one(double old, double nw, double eps, double eps_abs) {
    if (!isfinite(old)) return 0;
    const double delta = fabs(nw - old);
    return delta == 0.0 || delta < eps * old + eps_abs;
}

static void update_vertex_all(int64_t v, const double *xyz, const int64_t *row, const int32_t *oa,
                              const int32_t *ob, const double *d, double *out) {
    /* Reading: the new value is min(d_{k-1}(v), min over triangles of the
     * update step), so every d_k is monotone non-increasing in k. */
    double best = d[v];
    for (int64_t c = row[v]; c < row[v + 1]; ++c) {
        const double u = or_update(xyz + 3 * v, xyz + 3 * (int64_t)oa[c], xyz + 3 * (int64_t)ob[c], d[oa[c]], d[ob[c]]);
        if (u < best) best = u;
    }
    *out = best;
}

/*
 * PTP (Sec. 4.2).  Iteration k (k = 1, 2, ...) recomputes every non-source
 * vertex of the band B = V_{i_{k-1}} u ... u V_{j_k} from d_{k-1} only
 * (Jacobi: each vertex's new value depends on the previous map alone),
 * then sets the band bounds:
 *   j_k = k if k < rho else rho - 1                      (Eq. upper_band)
 *   i_k = i_{k-1} + 1 if every v in V_{i_{k-1}} passes the relative-change
 *         test, else i_{k-1}                               (Eq. lower_band)
 * and stops once i_k > rho - 1.  Readings: the band of iteration k runs from
 * the previous lower bound i_{k-1} (i_k is defined from d_k, so it cannot
 * bound the band that produces d_k); i_0 = 0 with the sources fixed at 0,
 * so V_0 always passes the test; vertices unreachable from S stay +inf.
 *
 * Outputs: d_out[n]; stats[4] = {K, rho, vertex updates, status}.
 * Optional traces (any pointer may be NULL), for the first trace_cap
 * iterations: trace_i[k-1] = i_{k-1} (the band's lower bound used at k),
 * trace_j[k-1] = j_k, trace_maxrel[k-1] = max relative change on V_{i_{k-1}}.
 * Optional history: d_hist[k*n + v] = d_k(v) for k = 0 .. hist_cap-1.
 * max_iter <= 0 means 8*rho + 64.
 * band_mode 1 replaces Eq. lower_band by the fixed band of the complexity
 * analysis (Sec. 6.1: the band holds the last k/2 toplesets), i.e. the lower
 * bound after iteration k is ceil(k/2), with no convergence test.
 * Returns OR_OK, OR_NOT_CONVERGED (max_iter reached, d_out still written)
 * or a negative error.
 */
int or_ptp(int64_t n, const double *xyz, int64_t nf, const int32_t *faces, int32_t m,
           const int32_t *src, double eps, double eps_abs, int64_t max_iter, int band_mode, double *d_out,
           int64_t *stats, int32_t *trace_i, int32_t *trace_j, double *trace_maxrel,
           int64_t trace_cap, double *d_hist, int64_t hist_cap) {
    if (n <= 0 || nf <= 0 || m <= 0 || !xyz || !faces || !src || !d_out) return OR_ERR_ARG;
    int64_t *row = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *oa = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * nf));
    int32_t *ob = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * nf));
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!row || !oa || !ob || !level) {
        free(row); free(oa); free(ob); free(level);
        return OR_ERR_NOMEM;
    }
    int rc = or_incident(n, nf, faces, row, oa, ob);
    if (rc != OR_OK) {
        free(row); free(oa); free(ob); free(level);
        return rc;
    }
    const int64_t rho = or_toplesets(n, row, oa, ob, m, src, level);
    if (rho < 0) {
        free(row); free(oa); free(ob); free(level);
        return (int)rho;
    }

    /* bucket the reachable vertices by topleset: V_r = order[off[r] .. off[r+1]-1] */
    int64_t *off = (int64_t *)calloc((size_t)(rho + 1), sizeof(int64_t));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *dn = (double *)malloc(sizeof(double) * (size_t)n);
    char *is_src = (char *)calloc((size_t)n, 1);
    if (!off || !order || !d || !dn || !is_src) {
        free(row); free(oa); free(ob); free(level); free(off); free(order); free(d); free(dn); free(is_src);
        return OR_ERR_NOMEM;
    }
    for (int64_t v = 0; v < n; ++v)
        if (level[v] >= 0) off[level[v] + 1] += 1;
    for (int64_t r = 0; r < rho; ++r) off[r + 1] += off[r];
    {
        int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rho + 1));
        memcpy(pos, off, sizeof(int64_t) * (size_t)(rho + 1));
        for (int64_t v = 0; v < n; ++v)
            if (level[v] >= 0) order[pos[level[v]]++] = v;
        free(pos);
    }

    /* d_0: +inf everywhere, 0 on S */
    for (int64_t v = 0; v < n; ++v) d[v] = INFINITY;
    for (int32_t s = 0; s < m; ++s) {
        d[src[s]] = 0.0;
        is_src[src[s]] = 1;
    }
    if (d_hist && hist_cap > 0) memcpy(d_hist, d, sizeof(double) * (size_t)n);

    if (max_iter <= 0) max_iter = 8 * rho + 64;
    int64_t i = 0, k = 0, updates = 0;
    int status = OR_NOT_CONVERGED;
    for (k = 1; k <= max_iter; ++k) {
        const int64_t j = k < rho ? k : rho - 1;
        const int64_t lo = off[i], hi = off[j + 1];
        /* Jacobi step on the band: new values from d_{k-1} only */
        for (int64_t q = lo; q < hi; ++q) {
            const int64_t v = order[q];
            if (is_src[v]) {
                dn[q] = d[v];
            } else {
                update_vertex_all(v, xyz, row, oa, ob, d, &dn[q]);
                updates += 1;
            }
        }
        /* relative-change test on V_{i_{k-1}} */
        int conv = 1;
        double maxrel = 0.0;
        for (int64_t q = off[i]; q < off[i + 1]; ++q) {
            const int64_t v = order[q];
            if (is_src[v]) continue;
            if (!converged_one(d[v], dn[q], eps, eps_abs)) conv = 0;
            const double rel = isfinite(d[v]) ? (d[v] > 0.0 ? fabs(dn[q] - d[v]) / d[v] : 0.0) : INFINITY;
            if (rel > maxrel) maxrel = rel;
        }
        /* commit d_k on the band; vertices outside it keep d_{k-1} */
        for (int64_t q = lo; q < hi; ++q) d[order[q]] = dn[q];
        if (k - 1 < trace_cap) {
            if (trace_i) trace_i[k - 1] = (int32_t)i;
            if (trace_j) trace_j[k - 1] = (int32_t)j;
            if (trace_maxrel) trace_maxrel[k - 1] = maxrel;
        }
        if (d_hist && k < hist_cap) memcpy(d_hist + (size_t)k * (size_t)n, d, sizeof(double) * (size_t)n);
        if (band_mode == 1) conv = (k + 1) / 2 > i;
        if (conv) i += 1;
        if (i > rho - 1) {
            status = OR_OK;
            break;
        }
    }
    if (k > max_iter) k = max_iter;
    memcpy(d_out, d, sizeof(double) * (size_t)n);
    if (stats) {
        stats[0] = k;
        stats[1] = rho;
        stats[2] = updates;
        stats[3] = status;
    }
    free(row); free(oa); free(ob); free(level); free(off); free(order); free(d); free(dn); free(is_src);
    return status;
}

/* splitmix64, used only to shuffle the sweep order in or_relax */
static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * Full relaxation without toplesets or band, to the fixpoint of the update
 * operator: repeat sweeps over all non-source vertices until a sweep changes
 * nothing.  mode 0: Jacobi (every vertex from the previous sweep's map);
 * mode 1: Gauss-Seidel in index order (in place); mode 2: in place, in a
 * fresh seeded random order every sweep.  Used to check that the update
 * operator's fixpoint does not depend on the update order.
 * Returns the number of sweeps, or a negative error.
 */
int64_t or_relax(int64_t n, const double *xyz, int64_t nf, const int32_t *faces, int32_t m,
                 const int32_t *src, int mode, uint64_t seed, int64_t max_sweeps, double *d_out) {
    if (n <= 0 || nf <= 0 || m <= 0 || !xyz || !faces || !src || !d_out) return OR_ERR_ARG;
    int64_t *row = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *oa = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * nf));
    int32_t *ob = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * nf));
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *dn = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    char *is_src = (char *)calloc((size_t)n, 1);
    int rc = (row && oa && ob && d && dn && perm && is_src) ? OR_OK : OR_ERR_NOMEM;
    if (rc == OR_OK) rc = or_incident(n, nf, faces, row, oa, ob);
    for (int32_t s = 0; rc == OR_OK && s < m; ++s)
        if (src[s] < 0 || src[s] >= n) rc = OR_ERR_INDEX;
    int64_t sweeps = 0;
    if (rc == OR_OK) {
        for (int64_t v = 0; v < n; ++v) d[v] = INFINITY;
        for (int32_t s = 0; s < m; ++s) {
            d[src[s]] = 0.0;
            is_src[src[s]] = 1;
        }
        for (int64_t v = 0; v < n; ++v) perm[v] = v;
        uint64_t state = seed;
        for (sweeps = 1; sweeps <= max_sweeps; ++sweeps) {
            int changed = 0;
            if (mode == 2) {
                for (int64_t q = n - 1; q > 0; --q) {
                    const int64_t r = (int64_t)(splitmix64(&state) % (uint64_t)(q + 1));
                    const int64_t t = perm[q];
                    perm[q] = perm[r];
                    perm[r] = t;
                }
            }
            if (mode == 0) {
                for (int64_t v = 0; v < n; ++v) {
                    if (is_src[v]) dn[v] = d[v];
                    else update_vertex_all(v, xyz, row, oa, ob, d, &dn[v]);
                }
                for (int64_t v = 0; v < n; ++v) {
                    if (dn[v] != d[v]) changed = 1;
                    d[v] = dn[v];
                }
            } else {
                for (int64_t q = 0; q < n; ++q) {
                    const int64_t v = perm[q];
                    if (is_src[v]) continue;
                    double nv;
                    update_vertex_all(v, xyz, row, oa, ob, d, &nv);
                    if (nv != d[v]) changed = 1;
                    d[v] = nv;
                }
            }
            if (!changed) break;
        }
        memcpy(d_out, d, sizeof(double) * (size_t)n);
    }
    free(row); free(oa); free(ob); free(d); free(dn); free(perm); free(is_src);
    return rc == OR_OK ? sweeps : rc;
}
