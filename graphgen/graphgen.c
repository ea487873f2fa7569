/*
 * Seeded synthetic graph generators (CSR, undirected, no self-loops, no
 * parallel edges).  This module holds none of the partitioning method's
 * arithmetic: it only produces inputs that both the oracle and the CUDA
 * library consume.  Every random draw comes from splitmix64 (Steele, Lea,
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014;
 * finaliser constants as published by Vigna) used as a counter-based
 * generator, so a graph is a pure function of its parameters and seed and is
 * identical on x86-64 and AArch64 hosts.
 *
 * Shapes follow the paper's synthetic workloads (Sec. 5, "Test Graphs": a
 * rectangular and a cubic mesh) and the usual stand-ins for its irregular
 * classes (R-MAT power-law graphs, random geometric graphs).
 *
 * All functions return 0 on success, nonzero on allocation failure.  Output
 * arrays are malloc'ed here and released with gg_free().
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

static inline uint64_t gg_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Independent stream per (seed, tag): tag separates vertex weights, edge
 * weights, R-MAT bits, permutations, ... */
static inline uint64_t gg_stream(uint64_t seed, uint64_t tag)
{
    return gg_splitmix64(seed ^ gg_splitmix64(tag * 0xD6E8FEB86659FD93ULL + 0x1234567ULL));
}

static inline uint64_t gg_draw(uint64_t stream, uint64_t counter)
{
    return gg_splitmix64(stream ^ gg_splitmix64(counter));
}

void gg_free(void *p) { free(p); }

/* uniform integer in [lo, hi] from a 64-bit draw (hi-lo+1 is tiny, bias is
 * below 2^-58 and irrelevant for synthetic inputs) */
static inline int32_t gg_uniform(uint64_t r, int32_t lo, int32_t hi)
{
    uint64_t span = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
    return (int32_t)((int64_t)lo + (int64_t)(r % span));
}

/* Weight of undirected edge {a, b}: drawn once per edge from the unordered
 * pair and mirrored to both CSR entries. */
static inline int32_t gg_edge_weight(uint64_t es, int64_t a, int64_t b, int32_t lo, int32_t hi)
{
    int64_t x = a < b ? a : b, y = a < b ? b : a;
    return gg_uniform(gg_draw(es, ((uint64_t)x << 32) ^ (uint64_t)y ^ ((uint64_t)x >> 32)), lo, hi);
}

/*
 * d-dimensional mesh with a (2d+1)-point stencil, d in {2, 3}: vertex id
 * x + nx*(y + ny*z); rows list neighbours in ascending id.  Vertex weights
 * uniform in [vlo, vhi], edge weights uniform in [elo, ehi] (lo == hi gives
 * constant weights).
 */
int gg_grid(int32_t nx, int32_t ny, int32_t nz, int32_t vlo, int32_t vhi,
            int32_t elo, int32_t ehi, uint64_t seed,
            int32_t *n_out, int64_t **xadj_out, int32_t **adjncy_out,
            int32_t **vwgt_out, int32_t **adjwgt_out)
{
    int64_t n = (int64_t)nx * ny * nz;
    int64_t *xadj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *vwgt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!xadj || !vwgt) { free(xadj); free(vwgt); return 1; }
    uint64_t vs = gg_stream(seed, 1), es = gg_stream(seed, 2);
    xadj[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t x = v % nx, y = (v / nx) % ny, z = v / ((int64_t)nx * ny);
        int d = (x > 0) + (x < nx - 1) + (y > 0) + (y < ny - 1) + (z > 0) + (z < nz - 1);
        xadj[v + 1] = xadj[v] + d;
        vwgt[v] = (vlo == vhi) ? vlo : gg_uniform(gg_draw(vs, (uint64_t)v), vlo, vhi);
    }
    int64_t nnz = xadj[n];
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t *ew = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!adj || !ew) { free(xadj); free(vwgt); free(adj); free(ew); return 1; }
    int64_t sxy = (int64_t)nx * ny;
    for (int64_t v = 0; v < n; ++v) {
        int64_t x = v % nx, y = (v / nx) % ny, z = v / sxy;
        int64_t j = xadj[v];
        int64_t nb[6]; int c = 0;
        if (z > 0) nb[c++] = v - sxy;
        if (y > 0) nb[c++] = v - nx;
        if (x > 0) nb[c++] = v - 1;
        if (x < nx - 1) nb[c++] = v + 1;
        if (y < ny - 1) nb[c++] = v + nx;
        if (z < nz - 1) nb[c++] = v + sxy;
        for (int i = 0; i < c; ++i) {
            adj[j + i] = (int32_t)nb[i];
            ew[j + i] = (elo == ehi) ? elo : gg_edge_weight(es, v, nb[i], elo, ehi);
        }
    }
    *n_out = (int32_t)n; *xadj_out = xadj; *adjncy_out = adj; *vwgt_out = vwgt; *adjwgt_out = ew;
    return 0;
}

/* ---- edge list -> CSR (symmetrise, drop self-loops, deduplicate) -------- */

static void gg_sort_row(int32_t *a, int64_t len)
{
    /* insertion sort for short rows, heap sort otherwise (no recursion) */
    if (len <= 32) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t x = a[i]; int64_t j = i - 1;
            while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
            a[j + 1] = x;
        }
        return;
    }
    for (int64_t start = len / 2 - 1; start >= 0; --start) {
        int64_t r = start;
        for (;;) {
            int64_t c = 2 * r + 1; if (c >= len) break;
            if (c + 1 < len && a[c + 1] > a[c]) ++c;
            if (a[r] >= a[c]) break;
            int32_t t = a[r]; a[r] = a[c]; a[c] = t; r = c;
        }
    }
    for (int64_t end = len - 1; end > 0; --end) {
        int32_t t = a[0]; a[0] = a[end]; a[end] = t;
        int64_t r = 0;
        for (;;) {
            int64_t c = 2 * r + 1; if (c >= end) break;
            if (c + 1 < end && a[c + 1] > a[c]) ++c;
            if (a[r] >= a[c]) break;
            int32_t t2 = a[r]; a[r] = a[c]; a[c] = t2; r = c;
        }
    }
}

/* Builds a symmetric CSR from directed pairs (src[i], dst[i]).  Self-loops
 * are dropped and duplicates merged; edge weights are drawn per unordered
 * pair.  src/dst are consumed (freed). */
static int gg_edges_to_csr(int64_t n, int64_t ne, int32_t *src, int32_t *dst,
                           int32_t vlo, int32_t vhi, int32_t elo, int32_t ehi, uint64_t seed,
                           int32_t *n_out, int64_t **xadj_out, int32_t **adjncy_out,
                           int32_t **vwgt_out, int32_t **adjwgt_out)
{
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return 1;
    for (int64_t i = 0; i < ne; ++i) if (src[i] != dst[i]) { deg[src[i]]++; deg[dst[i]]++; }
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!off) { free(deg); return 1; }
    off[0] = 0;
    for (int64_t v = 0; v < n; ++v) off[v + 1] = off[v] + deg[v];
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(off[n] > 0 ? off[n] : 1));
    if (!tmp) { free(deg); free(off); return 1; }
    memcpy(deg, off, sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < ne; ++i) {
        int32_t a = src[i], b = dst[i];
        if (a == b) continue;
        tmp[deg[a]++] = b; tmp[deg[b]++] = a;
    }
    free(src); free(dst);
    /* sort + dedup each row in place, record new lengths */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v) {
        int32_t *row = tmp + off[v]; int64_t len = off[v + 1] - off[v];
        gg_sort_row(row, len);
        int64_t w = 0;
        for (int64_t i = 0; i < len; ++i) if (w == 0 || row[i] != row[w - 1]) row[w++] = row[i];
        deg[v] = w;
    }
    int64_t *xadj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!xadj) { free(deg); free(off); free(tmp); return 1; }
    xadj[0] = 0;
    for (int64_t v = 0; v < n; ++v) xadj[v + 1] = xadj[v] + deg[v];
    int64_t nnz = xadj[n];
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t *ew = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t *vw = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!adj || !ew || !vw) { free(deg); free(off); free(tmp); free(xadj); free(adj); free(ew); free(vw); return 1; }
    uint64_t vs = gg_stream(seed, 1), es = gg_stream(seed, 2);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v) {
        memcpy(adj + xadj[v], tmp + off[v], sizeof(int32_t) * (size_t)deg[v]);
        for (int64_t j = xadj[v]; j < xadj[v + 1]; ++j)
            ew[j] = (elo == ehi) ? elo : gg_edge_weight(es, v, adj[j], elo, ehi);
        vw[v] = (vlo == vhi) ? vlo : gg_uniform(gg_draw(vs, (uint64_t)v), vlo, vhi);
    }
    free(deg); free(off); free(tmp);
    *n_out = (int32_t)n; *xadj_out = xadj; *adjncy_out = adj; *vwgt_out = vw; *adjwgt_out = ew;
    return 0;
}

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): 2^scale vertices,
 * edge_factor * 2^scale generated directed edges, recursive quadrant
 * probabilities (a, b, c, 1-a-b-c).  Vertex labels are then shuffled with a
 * seeded Fisher-Yates permutation (as the Graph500 generator does) so that
 * degree does not correlate with id.  Isolated vertices are kept.
 */
int gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed,
            int32_t vlo, int32_t vhi, int32_t elo, int32_t ehi,
            int32_t *n_out, int64_t **xadj_out, int32_t **adjncy_out,
            int32_t **vwgt_out, int32_t **adjwgt_out)
{
    int64_t n = (int64_t)1 << scale;
    int64_t ne = (int64_t)edge_factor * n;
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)ne);
    int32_t *dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)ne);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!src || !dst || !perm) { free(src); free(dst); free(perm); return 1; }
    /* thresholds on 53-bit integers: deterministic on every IEEE host */
    const double two53 = 9007199254740992.0;
    uint64_t ta = (uint64_t)(a * two53), tb = (uint64_t)((a + b) * two53), tc = (uint64_t)((a + b + c) * two53);
    uint64_t rs = gg_stream(seed, 3);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) {
        int64_t s = 0, d = 0;
        for (int32_t l = 0; l < scale; ++l) {
            uint64_t r = gg_draw(rs, (uint64_t)e * (uint64_t)scale + (uint64_t)l) >> 11;
            int sb, db;
            if (r < ta) { sb = 0; db = 0; }
            else if (r < tb) { sb = 0; db = 1; }
            else if (r < tc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            s = (s << 1) | sb; d = (d << 1) | db;
        }
        src[e] = (int32_t)s; dst[e] = (int32_t)d;
    }
    uint64_t ps = gg_stream(seed, 4);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)(gg_draw(ps, (uint64_t)i) % (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) { src[e] = perm[src[e]]; dst[e] = perm[dst[e]]; }
    free(perm);
    return gg_edges_to_csr(n, ne, src, dst, vlo, vhi, elo, ehi, seed,
                           n_out, xadj_out, adjncy_out, vwgt_out, adjwgt_out);
}

/*
 * Random geometric graph in the unit square: n points drawn uniformly,
 * an edge between every pair closer than radius.  Cell-list neighbour search.
 */
int gg_rgg(int32_t n, double radius, uint64_t seed, int32_t vlo, int32_t vhi, int32_t elo, int32_t ehi,
           int32_t *n_out, int64_t **xadj_out, int32_t **adjncy_out,
           int32_t **vwgt_out, int32_t **adjwgt_out)
{
    double *px = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *py = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!px || !py) { free(px); free(py); return 1; }
    uint64_t s = gg_stream(seed, 5);
    for (int64_t v = 0; v < n; ++v) {
        px[v] = (double)(gg_draw(s, 2 * (uint64_t)v) >> 11) * (1.0 / 9007199254740992.0);
        py[v] = (double)(gg_draw(s, 2 * (uint64_t)v + 1) >> 11) * (1.0 / 9007199254740992.0);
    }
    int64_t g = (int64_t)floor(1.0 / radius); if (g < 1) g = 1; if (g > 4096) g = 4096;
    int64_t ncell = g * g;
    int64_t *cstart = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    int32_t *cidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!cstart || !cidx) { free(px); free(py); free(cstart); free(cidx); return 1; }
    for (int64_t v = 0; v < n; ++v) {
        int64_t cx = (int64_t)(px[v] * g), cy = (int64_t)(py[v] * g);
        if (cx >= g) cx = g - 1; if (cy >= g) cy = g - 1;
        cstart[cy * g + cx + 1]++;
    }
    for (int64_t i = 0; i < ncell; ++i) cstart[i + 1] += cstart[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    if (!fill) { free(px); free(py); free(cstart); free(cidx); return 1; }
    memcpy(fill, cstart, sizeof(int64_t) * (size_t)ncell);
    for (int64_t v = 0; v < n; ++v) {
        int64_t cx = (int64_t)(px[v] * g), cy = (int64_t)(py[v] * g);
        if (cx >= g) cx = g - 1; if (cy >= g) cy = g - 1;
        cidx[fill[cy * g + cx]++] = (int32_t)v;
    }
    free(fill);
    double r2 = radius * radius;
    /* two passes: count, then emit directed pairs u<v */
    int64_t cnt = 0;
    for (int pass = 0; pass < 2; ++pass) {
        int32_t *src = NULL, *dst = NULL;
        if (pass == 1) {
            src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
            dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
            if (!src || !dst) { free(src); free(dst); free(px); free(py); free(cstart); free(cidx); return 1; }
        }
        int64_t e = 0;
        for (int64_t cy = 0; cy < g; ++cy)
            for (int64_t cx = 0; cx < g; ++cx)
                for (int64_t i = cstart[cy * g + cx]; i < cstart[cy * g + cx + 1]; ++i) {
                    int32_t v = cidx[i];
                    for (int64_t dy = -1; dy <= 1; ++dy)
                        for (int64_t dx = -1; dx <= 1; ++dx) {
                            int64_t qx = cx + dx, qy = cy + dy;
                            if (qx < 0 || qy < 0 || qx >= g || qy >= g) continue;
                            for (int64_t jj = cstart[qy * g + qx]; jj < cstart[qy * g + qx + 1]; ++jj) {
                                int32_t u = cidx[jj];
                                if (u <= v) continue;
                                double ddx = px[u] - px[v], ddy = py[u] - py[v];
                                if (ddx * ddx + ddy * ddy < r2) {
                                    if (pass == 1) { src[e] = v; dst[e] = u; }
                                    ++e;
                                }
                            }
                        }
                }
        if (pass == 0) cnt = e;
        else {
            free(px); free(py); free(cstart); free(cidx);
            return gg_edges_to_csr(n, cnt, src, dst, vlo, vhi, elo, ehi, seed,
                                   n_out, xadj_out, adjncy_out, vwgt_out, adjwgt_out);
        }
    }
    return 1;
}

/* Erdos-Renyi G(n, p) for small test graphs (pairs tested in order). */
int gg_gnp(int32_t n, double p, uint64_t seed, int32_t vlo, int32_t vhi, int32_t elo, int32_t ehi,
           int32_t *n_out, int64_t **xadj_out, int32_t **adjncy_out,
           int32_t **vwgt_out, int32_t **adjwgt_out)
{
    uint64_t s = gg_stream(seed, 6);
    const double two53 = 9007199254740992.0;
    uint64_t tp = (uint64_t)(p * two53);
    int64_t cnt = 0;
    for (int64_t v = 0; v < n; ++v)
        for (int64_t u = v + 1; u < n; ++u)
            if ((gg_draw(s, (uint64_t)v * (uint64_t)n + (uint64_t)u) >> 11) < tp) ++cnt;
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
    int32_t *dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
    if (!src || !dst) { free(src); free(dst); return 1; }
    int64_t e = 0;
    for (int64_t v = 0; v < n; ++v)
        for (int64_t u = v + 1; u < n; ++u)
            if ((gg_draw(s, (uint64_t)v * (uint64_t)n + (uint64_t)u) >> 11) < tp) { src[e] = (int32_t)v; dst[e] = (int32_t)u; ++e; }
    return gg_edges_to_csr(n, cnt, src, dst, vlo, vhi, elo, ehi, seed,
                           n_out, xadj_out, adjncy_out, vwgt_out, adjwgt_out);
}

/* CSR from caller-given undirected edge list (copied). */
int gg_from_edges(int32_t n, int64_t ne, const int32_t *src_in, const int32_t *dst_in,
                  int32_t vlo, int32_t vhi, int32_t elo, int32_t ehi, uint64_t seed,
                  int32_t *n_out, int64_t **xadj_out, int32_t **adjncy_out,
                  int32_t **vwgt_out, int32_t **adjwgt_out)
{
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne > 0 ? ne : 1));
    int32_t *dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne > 0 ? ne : 1));
    if (!src || !dst) { free(src); free(dst); return 1; }
    if (ne > 0) { memcpy(src, src_in, sizeof(int32_t) * (size_t)ne); memcpy(dst, dst_in, sizeof(int32_t) * (size_t)ne); }
    return gg_edges_to_csr(n, ne, src, dst, vlo, vhi, elo, ehi, seed,
                           n_out, xadj_out, adjncy_out, vwgt_out, adjwgt_out);
}
