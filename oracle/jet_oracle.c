/*
 * ORACLE — test infrastructure, not product code.
 *
 * A plain, slow, single-threaded CPU statement of what the Jet partitioner
 * computes (Gilbert, Madduri, Boman, Rajamanickam, "Jet: Multilevel Graph
 * Partitioning on Graphics Processing Units").  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the CUDA
 * library never does, and the two share no code.  Every function follows one
 * passage of the paper, cited in its comment; where the paper leaves a value
 * open, the reading taken is stated at that point (and listed, with all the
 * others, in the design notes).
 *
 * Conventions (Sec. 2.1 "Problem Definition"): undirected CSR graph without
 * self-loops or parallel edges, xadj int64[n+1], adjncy int32[xadj[n]],
 * positive integer vertex weights vwgt and symmetric edge weights adjwgt
 * (NULL means unit weights).  Sums (part weights, cut, prefixes) are int64;
 * connectivities and gains are int64 here.
 *
 * Parity status: every function is pinned by the CPU tests (brute force on
 * tiny graphs, hand-derived fixtures, closed forms and the paper's stated
 * invariants); none is "parity unpinned".
 */
#define _POSIX_C_SOURCE 200809L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <time.h>

#define OR_NONE INT64_MIN /* "negative infinity" gain of Alg. 4 */

typedef struct {
    int32_t n;
    const int64_t *xadj;
    const int32_t *adjncy;
    const int32_t *vwgt;   /* NULL: unit */
    const int32_t *adjwgt; /* NULL: unit */
} or_graph;

/* Hyper-parameters named by the paper, with its defaults (Sec. 4, 4.1.2, 4.2.2,
 * Sec. 3).  c and phi are held as exact rationals so that every decision is
 * an integer comparison. */
typedef struct {
    int32_t c_fine_q16;     /* c on the finest level  * 65536 (0.25 -> 16384), Sec. 4.1.2 */
    int32_t c_coarse_q16;   /* c on the other levels * 65536 (0.75 -> 49152) */
    int32_t phi_ppm;        /* phi * 1e6 (0.999 -> 999000), Alg. 3 tolerance check */
    int32_t max_no_improve; /* 12 iterations without a new best, Sec. 4 */
    int32_t weak_limit;     /* b_max = 2 Jetrw iterations, then Jetrs, Sec. 4.2.2 */
    int32_t coarsen_target; /* 0: max(8k, 256) vertices (Sec. 3: "between 4k and 8k") */
    int32_t max_levels;     /* hierarchy depth cap (64) */
    int32_t max_iters;      /* per-level safety cap on refinement iterations (10000) */
    int32_t hem_rounds;     /* heavy-edge matching rounds (8) */
    int32_t flags;          /* ablation switches, OR_ABL_* */
} or_opts;

/* Jetlp ablation switches (Sec. 6.1.4 "Component Effectiveness", Table 2) */
#define OR_ABL_NO_LOCKS      1 /* ignore the lock bit */
#define OR_ABL_NO_AFTERBURN  2 /* M = X (no second filter) */
#define OR_ABL_WEAK_AFTERBURN 4 /* first filter keeps only F >= 0 */
#define OR_ABL_BASELINE_LP   8 /* baseline LP: move iff F > 0, no afterburner, no locks */
#define OR_ABL_STRICT_GAIN  32 /* first filter keeps only F > 0 (with NO_AFTERBURN: the baseline plus locks) */
/* Coarsening switch (Sec. 3.1): add two-hop matches after heavy-edge matching.
 * Off in the plain method, whose coarsening is heavy-edge matching alone. */
#define OR_TWO_HOP          16

typedef struct {
    int32_t levels;
    int64_t n[64], m[64];
    int32_t it_lp[64], it_rw[64], it_rs[64];
    int64_t cut_level[64];   /* cut of P_best after refining level i */
    int64_t edge_iters;      /* sum over levels of iterations * m_level */
    int64_t fin_edge_iters;  /* the same, finest level only */
    int64_t cut, maxw;
    double sec_coarsen, sec_init, sec_refine, sec_refine_finest;
} or_stats;

static double or_now(void)
{
    struct timespec ts; clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static inline int64_t vw(const or_graph *g, int64_t v) { return g->vwgt ? g->vwgt[v] : 1; }
static inline int64_t ew(const or_graph *g, int64_t j) { return g->adjwgt ? g->adjwgt[j] : 1; }

void or_free(void *p) { free(p); }

/* splitmix64 as published (Steele, Lea, Flood 2014; Vigna's constants). */
uint64_t or_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1: cost (cutsize) and part weights                           */
/* ------------------------------------------------------------------ */

/* cutsize = sum of weights of edges whose endpoints lie in different parts;
 * every undirected edge appears twice in CSR, hence the halving. */
int64_t or_cut(const or_graph *g, const int32_t *part)
{
    int64_t twice = 0;
    for (int64_t v = 0; v < g->n; ++v)
        for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; ++j)
            if (part[g->adjncy[j]] != part[v]) twice += ew(g, j);
    return twice / 2;
}

/* weight(p_i) = sum of the weights of its vertices */
void or_part_weights(const or_graph *g, const int32_t *part, int32_t k, int64_t *pw)
{
    for (int32_t p = 0; p < k; ++p) pw[p] = 0;
    for (int64_t v = 0; v < g->n; ++v) pw[part[v]] += vw(g, v);
}

static int64_t or_maxw(const int64_t *pw, int32_t k)
{
    int64_t m = 0;
    for (int32_t p = 0; p < k; ++p) if (pw[p] > m) m = pw[p];
    return m;
}

/* Balance constraint, Sec. 2.1: weight(p) <= (1+lambda) W / k.  Reading
 * (the paper does not say how the real bound is rounded): opt = ceil(W/k),
 * L = floor(opt * (10^6 + e) / 10^6) with e = round(lambda * 10^6). */
int64_t or_limit(int64_t W, int32_t k, double eps, int64_t *opt_out)
{
    int64_t opt = (W + k - 1) / k;
    int64_t e = llround(eps * 1e6);
    if (opt_out) *opt_out = opt;
    return opt * (1000000 + e) / 1000000;
}

/* sigma = maxDestSize (Alg. 5): the paper only asks for a dead zone between
 * valid destinations and oversized parts.  Reading: the middle of the
 * tolerance, opt + floor((L - opt) / 2), so that a destination may overshoot
 * sigma by half the tolerance before it becomes oversized. */
int64_t or_sigma(int64_t opt, int64_t L) { return opt + (L - opt) / 2; }

/* slot() of Sec. 4.2.1: 0 for negative loss, 1 for zero, 2 + floor(log2 x) */
int32_t or_slot(int64_t x)
{
    if (x < 0) return 0;
    if (x == 0) return 1;
    int32_t l = 0;
    while (x > 1) { x >>= 1; ++l; }
    return 2 + l;
}

/* conn(v, p) for all p adjacent to v (the quantity the paper's hash-table
 * data structure of Sec. 4.3 caches).  Fills the dense table conn[] for the
 * touched parts and lists them; caller resets with conn_reset(). */
static int32_t conn_gather(const or_graph *g, const int32_t *part, int64_t v, int64_t *conn, int32_t *touched)
{
    int32_t cnt = 0;
    for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; ++j) {
        int32_t p = part[g->adjncy[j]];
        if (conn[p] == 0) touched[cnt++] = p;
        conn[p] += ew(g, j);
    }
    return cnt;
}

static void conn_reset(int64_t *conn, const int32_t *touched, int32_t cnt)
{
    for (int32_t i = 0; i < cnt; ++i) conn[touched[i]] = 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.1, Alg. 4: Jetlp                                             */
/* ------------------------------------------------------------------ */

/*
 * One Jetlp pass on partition P with lock set R (locked[v] != 0).
 *  - destination (Eq. for P_d): P_d(v) = argmax_{p != P_s(v)} conn(v, p) over
 *    the parts adjacent to v, ties to the lowest part id (the paper's ties are
 *    racy, Sec. 4.3; this is the fixed rule); F(v) = conn(v,P_d) - conn(v,P_s);
 *    F = -inf when v is locked or only adjacent to its own part.
 *  - first filter (Eq. gainconn_filter): v in X iff F(v) != -inf and
 *    (F(v) >= 0 or -F(v) < floor(c * conn(v, P_s))).
 *  - afterburner (Alg. 4 second loop, ord of Sec. 4.1.1): for v in X,
 *    F2(v) = sum over neighbours u of w * ([p_u = P_d(v)] - [p_u = P_s(v)]),
 *    p_u = P_d(u) if u in X and (F(u) > F(v) or (F(u) = F(v) and u < v)),
 *    else P_s(u).
 *  - second filter: M = {v in X : F2(v) >= 0}.
 * Outputs per vertex: Pd, F (OR_NONE for -inf), inX, F2 (0 outside X), inM.
 * abl: OR_ABL_* switches (0 = the full Jetlp).
 */
void or_jetlp(const or_graph *g, int32_t k, const int32_t *P, const uint8_t *locked, int32_t c_q16,
              int32_t abl, int32_t *Pd, int64_t *F, uint8_t *inX, int64_t *F2, uint8_t *inM)
{
    int64_t n = g->n;
    int64_t *conn = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    int64_t *conn_s = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int ignore_locks = (abl & (OR_ABL_NO_LOCKS | OR_ABL_BASELINE_LP)) != 0;
    for (int64_t v = 0; v < n; ++v) {
        Pd[v] = P[v]; F[v] = OR_NONE; conn_s[v] = 0;
        if (locked && locked[v] && !ignore_locks) continue;
        int32_t cnt = conn_gather(g, P, v, conn, touched);
        int32_t best = -1;
        for (int32_t i = 0; i < cnt; ++i) {
            int32_t p = touched[i];
            if (p == P[v]) continue;
            if (best < 0 || conn[p] > conn[best] || (conn[p] == conn[best] && p < best)) best = p;
        }
        conn_s[v] = conn[P[v]];
        if (best >= 0) { Pd[v] = best; F[v] = conn[best] - conn[P[v]]; }
        conn_reset(conn, touched, cnt);
    }
    for (int64_t v = 0; v < n; ++v) {
        int64_t f = F[v];
        int x = 0;
        if (f != OR_NONE) {
            if (abl & (OR_ABL_BASELINE_LP | OR_ABL_STRICT_GAIN)) x = f > 0;
            else if (abl & OR_ABL_WEAK_AFTERBURN) x = f >= 0;
            else x = (f >= 0) || (-f < (c_q16 * conn_s[v]) / 65536);
        }
        inX[v] = (uint8_t)x;
    }
    for (int64_t v = 0; v < n; ++v) {
        F2[v] = 0; inM[v] = 0;
        if (!inX[v]) continue;
        if (abl & (OR_ABL_NO_AFTERBURN | OR_ABL_BASELINE_LP)) { inM[v] = 1; continue; }
        int64_t f2 = 0;
        for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; ++j) {
            int32_t u = g->adjncy[j];
            int32_t pu = P[u];
            if (inX[u] && (F[u] > F[v] || (F[u] == F[v] && u < v))) pu = Pd[u];
            if (pu == Pd[v]) f2 += ew(g, j);
            else if (pu == P[v]) f2 -= ew(g, j);
        }
        F2[v] = f2;
        inM[v] = f2 >= 0;
    }
    free(conn); free(touched); free(conn_s);
}

/* ------------------------------------------------------------------ */
/* Sec. 4.2, Alg. 5: rebalancing (Jetrw, Jetrs)                         */
/* ------------------------------------------------------------------ */

typedef struct { int32_t slot; int32_t v; } or_cand;

static int cand_cmp(const void *a, const void *b)
{
    const or_cand *x = (const or_cand *)a, *y = (const or_cand *)b;
    if (x->slot != y->slot) return x->slot < y->slot ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

/*
 * Shared by Jetrw and Jetrs.  A = {p : w_p > L}, B = {p : w_p <= sigma}
 * (Alg. 5).  For every v in a part of A that may leave it (heavy-vertex
 * rule of Sec. 4.2.2: v stays if vwgt(v) > 1.5 (w_p - opt); integer form
 * 2 vwgt(v) > 3 (w_p - opt)), the caller's loss has already been stored in
 * loss[v] (and cand[v] = 1).  Eviction (Alg. 5 scan): per part of A, the
 * candidates in the order (slot(loss) ascending, vertex id ascending) — the
 * paper's order inside a slot is racy, this is the fixed one — are taken
 * while the weight taken before them is below w_p - L (reading: exclusive
 * prefix, so a part ends at or below L when enough weight is eligible).
 * Marks taken[v].
 */
static void or_evict(const or_graph *g, int32_t k, const int32_t *P, const int64_t *pw, int64_t L,
                     const uint8_t *cand, const int64_t *loss, uint8_t *taken)
{
    int64_t n = g->n;
    int64_t *cnt = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) { taken[v] = 0; if (cand[v]) cnt[P[v] + 1]++; }
    for (int32_t p = 0; p < k; ++p) cnt[p + 1] += cnt[p];
    or_cand *list = (or_cand *)malloc(sizeof(or_cand) * (size_t)(cnt[k] > 0 ? cnt[k] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    for (int32_t p = 0; p < k; ++p) fill[p] = cnt[p];
    for (int64_t v = 0; v < n; ++v)
        if (cand[v]) { list[fill[P[v]]].slot = or_slot(loss[v]); list[fill[P[v]]].v = (int32_t)v; fill[P[v]]++; }
    for (int32_t p = 0; p < k; ++p) {
        if (pw[p] <= L) continue;
        int64_t len = cnt[p + 1] - cnt[p];
        or_cand *lp = list + cnt[p];
        qsort(lp, (size_t)len, sizeof(or_cand), cand_cmp);
        int64_t excess = pw[p] - L, before = 0;
        for (int64_t i = 0; i < len; ++i) {
            if (before >= excess) break;
            taken[lp[i].v] = 1;
            before += vw(g, lp[i].v);
        }
    }
    free(cnt); free(list); free(fill);
}

static int or_may_leave(const or_graph *g, int64_t v, const int64_t *pw, const int32_t *P, int64_t opt)
{
    return 2 * vw(g, v) <= 3 * (pw[P[v]] - opt);
}

/*
 * Jetrw, Alg. 5 (weak rebalancing).  For each eligible v in an oversized
 * part: P_d(v) = argmax conn(v, p) over the adjacent parts in B, ties to the
 * lowest id; if v touches no part of B, P_d(v) = B[h mod |B|] with B in
 * ascending id and h = splitmix64(seed ^ (0x9E3779B97F4A7C15 (iter+1)) ^ v)
 * (reading of randomPart(B)); loss F(v) = conn(v,P_s) - conn(v,P_d) (the sign
 * of Alg. 5).  Evicted vertices move to P_d.  dest[v] = new part or -1.
 * Returns |M|; *ncand_out = number of candidates.
 */
int64_t or_jetrw(const or_graph *g, int32_t k, const int32_t *P, const int64_t *pw, int64_t L, int64_t opt,
                 int64_t sigma, uint64_t seed, int32_t iter, int32_t *dest, int64_t *loss_out, int64_t *ncand_out)
{
    int64_t n = g->n;
    int64_t *conn = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    int32_t *Bs = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    uint8_t *inB = (uint8_t *)calloc((size_t)k, 1);
    int32_t nB = 0;
    for (int32_t p = 0; p < k; ++p) if (pw[p] <= sigma) { Bs[nB++] = p; inB[p] = 1; }
    int64_t *loss = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    uint8_t *cand = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    uint8_t *taken = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int32_t *pd = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t ncand = 0;
    for (int64_t v = 0; v < n; ++v) {
        pd[v] = P[v];
        if (pw[P[v]] <= L || !or_may_leave(g, v, pw, P, opt) || nB == 0) continue;
        int32_t cnt = conn_gather(g, P, v, conn, touched);
        int32_t best = -1;
        for (int32_t i = 0; i < cnt; ++i) {
            int32_t p = touched[i];
            if (!inB[p]) continue;
            if (best < 0 || conn[p] > conn[best] || (conn[p] == conn[best] && p < best)) best = p;
        }
        int64_t cd = 0;
        if (best >= 0) cd = conn[best];
        else {
            uint64_t h = or_splitmix64(seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(iter + 1)) ^ (uint64_t)v);
            best = Bs[h % (uint64_t)nB];
        }
        pd[v] = best;
        loss[v] = conn[P[v]] - cd;
        cand[v] = 1; ++ncand;
        conn_reset(conn, touched, cnt);
    }
    or_evict(g, k, P, pw, L, cand, loss, taken);
    int64_t nm = 0;
    for (int64_t v = 0; v < n; ++v) {
        dest[v] = taken[v] ? pd[v] : -1;
        if (taken[v]) ++nm;
        if (loss_out) loss_out[v] = cand[v] ? loss[v] : OR_NONE;
    }
    if (ncand_out) *ncand_out = ncand;
    free(conn); free(touched); free(Bs); free(inB); free(loss); free(cand); free(taken); free(pd);
    return nm;
}

/*
 * Jetrs (Sec. 4.2.2, strong rebalancing).  Same A, B, sigma and eligibility.
 * loss(v) = conn(v,P_s) - floor(S_v / c_v), S_v = sum of conn(v,p) over the
 * parts p in B adjacent to v, c_v their number; floor(S/0) := 0 (reading: the
 * sign of Alg. 5, integer mean).  Eviction as in Jetrw.  The evicted list E
 * (the paper's "unordered list") is taken in ascending vertex id (reading);
 * s_e = weight of E before e.  Destinations b in B in ascending id get
 * capacity cap_b = sigma - w_b laid end to end ("cookie cutter"); e goes to
 * the b whose interval holds the middle of e, C_b <= s_e + w_e/2 < C_b +
 * cap_b (C_b = capacity before b; doubled to stay in integers), so that each
 * destination receives a weight as close to its capacity as the cuts allow;
 * e stays if its middle lies past the last capacity.  With unit weights this
 * is C_b <= s_e < C_b + cap_b.  dest[v] = new part or -1.  Returns |M|.
 */
int64_t or_jetrs(const or_graph *g, int32_t k, const int32_t *P, const int64_t *pw, int64_t L, int64_t opt,
                 int64_t sigma, int32_t *dest, int64_t *loss_out, int64_t *ncand_out)
{
    int64_t n = g->n;
    int64_t *conn = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    uint8_t *inB = (uint8_t *)calloc((size_t)k, 1);
    int32_t nB = 0;
    for (int32_t p = 0; p < k; ++p) if (pw[p] <= sigma) { inB[p] = 1; ++nB; }
    int64_t *loss = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    uint8_t *cand = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    uint8_t *taken = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t ncand = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (pw[P[v]] <= L || !or_may_leave(g, v, pw, P, opt) || nB == 0) continue;
        int32_t cnt = conn_gather(g, P, v, conn, touched);
        int64_t S = 0, c = 0;
        for (int32_t i = 0; i < cnt; ++i)
            if (inB[touched[i]]) { S += conn[touched[i]]; ++c; }
        loss[v] = conn[P[v]] - (c > 0 ? S / c : 0);
        cand[v] = 1; ++ncand;
        conn_reset(conn, touched, cnt);
    }
    or_evict(g, k, P, pw, L, cand, loss, taken);
    /* capacities of B in ascending part id, C_b = capacity before b */
    int64_t *C = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + 1));
    int32_t *Bs = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    int32_t nb = 0; int64_t tot = 0;
    for (int32_t p = 0; p < k; ++p) if (inB[p]) { Bs[nb] = p; C[nb] = tot; tot += sigma - pw[p]; ++nb; }
    C[nb] = tot;
    int64_t s = 0, nm = 0;
    for (int64_t v = 0; v < n; ++v) {
        dest[v] = -1;
        if (loss_out) loss_out[v] = cand[v] ? loss[v] : OR_NONE;
        if (!taken[v]) continue;
        int64_t mid2 = 2 * s + vw(g, v);
        for (int32_t i = 0; i < nb; ++i)
            if (2 * C[i] <= mid2 && mid2 < 2 * C[i + 1]) { dest[v] = Bs[i]; ++nm; break; }
        s += vw(g, v);
    }
    if (ncand_out) *ncand_out = ncand;
    free(conn); free(touched); free(inB); free(loss); free(cand); free(taken); free(C); free(Bs);
    return nm;
}

/* ------------------------------------------------------------------ */
/* Sec. 4, Alg. 3: Jet refinement driver                              */
/* ------------------------------------------------------------------ */

#define OR_KIND_LP 0
#define OR_KIND_RW 1
#define OR_KIND_RS 2

/*
 * Refines part_inout in place (Alg. 3) and returns its status (0 balanced,
 * 1 the best partition found is still unbalanced).
 *  - iteration: if max part weight <= L run Jetlp (locks R := M afterwards,
 *    weak counter := 0); else Jetrw while the weak counter is below b_max
 *    (counter += 1), else Jetrs.  Moves are applied synchronously.
 *  - P_best: starts at P_0.  A balanced P_iter replaces P_best if P_best is
 *    unbalanced or cost(P_iter) < cost(P_best); the no-improvement counter is
 *    reset if P_best was unbalanced or cost(P_iter) < phi cost(P_best) (Alg. 3
 *    tolerance check, phi exact as phi_ppm / 10^6).  An unbalanced P_iter
 *    replaces an unbalanced P_best with larger max part weight, and resets
 *    the counter (Alg. 3 ElsIf).  Reading: a balanced partition always
 *    replaces an unbalanced best.
 *  - stop when the counter reaches max_no_improve (12, Sec. 4) or after
 *    max_iters iterations (safety cap).
 * Cut and part weights are recomputed from scratch after every iteration.
 * c_q16: the first-filter ratio for this level.  seed: Jetrw's hash seed.
 * Trace arrays (may be NULL) receive per-iteration kind, |X| (Jetlp) or
 * number of rebalancing candidates, |M|, cut and max part weight.
 */
int or_refine(const or_graph *g, int32_t k, double eps, int32_t c_q16, uint64_t seed, const or_opts *o,
              int32_t *part_inout, int64_t *cut_out, int64_t *maxw_out,
              int32_t trace_cap, int32_t *tr_kind, int64_t *tr_nx, int64_t *tr_nm, int64_t *tr_cut,
              int64_t *tr_maxw, int32_t *iters_out, int32_t *kind_count)
{
    int64_t n = g->n;
    int64_t W = 0;
    for (int64_t v = 0; v < n; ++v) W += vw(g, v);
    int64_t opt = 0;
    int64_t L = or_limit(W, k, eps, &opt);
    int64_t sigma = or_sigma(opt, L);
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *P = part_inout;
    int32_t *Pbest = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *Pd = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *dest = (int32_t *)malloc(sizeof(int32_t) * nn);
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * nn);
    int64_t *F2 = (int64_t *)malloc(sizeof(int64_t) * nn);
    uint8_t *inX = (uint8_t *)malloc(nn), *inM = (uint8_t *)malloc(nn);
    uint8_t *locked = (uint8_t *)calloc(nn, 1);
    int64_t *pw = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    memcpy(Pbest, P, sizeof(int32_t) * (size_t)n);
    or_part_weights(g, P, k, pw);
    int64_t cut = or_cut(g, P), maxw = or_maxw(pw, k);
    int64_t best_cut = cut, best_maxw = maxw;
    int best_bal = maxw <= L;
    int32_t noimp = 0, weak = 0, it = 0;
    if (kind_count) kind_count[0] = kind_count[1] = kind_count[2] = 0;
    while (noimp < o->max_no_improve && it < o->max_iters) {
        int32_t kind;
        int64_t nx = 0, nm = 0;
        if (maxw <= L) {
            kind = OR_KIND_LP; weak = 0;
            or_jetlp(g, k, P, locked, c_q16, o->flags, Pd, F, inX, F2, inM);
            for (int64_t v = 0; v < n; ++v) {
                nx += inX[v];
                dest[v] = inM[v] ? Pd[v] : -1;
                nm += inM[v];
            }
        } else if (weak < o->weak_limit) {
            kind = OR_KIND_RW; weak++;
            nm = or_jetrw(g, k, P, pw, L, opt, sigma, seed, it, dest, NULL, &nx);
        } else {
            kind = OR_KIND_RS;
            nm = or_jetrs(g, k, P, pw, L, opt, sigma, dest, NULL, &nx);
        }
        for (int64_t v = 0; v < n; ++v) if (dest[v] >= 0) P[v] = dest[v];
        if (kind == OR_KIND_LP && !(o->flags & (OR_ABL_NO_LOCKS | OR_ABL_BASELINE_LP)))
            for (int64_t v = 0; v < n; ++v) locked[v] = inM[v];
        /* updatePartsAndDS: recomputed from scratch (the self-check) */
        or_part_weights(g, P, k, pw);
        cut = or_cut(g, P); maxw = or_maxw(pw, k);
        ++it; ++noimp;
        if (maxw <= L) {
            if (!best_bal || cut < best_cut) {
                if (!best_bal || (int64_t)1000000 * cut < (int64_t)o->phi_ppm * best_cut) noimp = 0;
                memcpy(Pbest, P, sizeof(int32_t) * (size_t)n);
                best_cut = cut; best_maxw = maxw; best_bal = 1;
            }
        } else if (!best_bal && maxw < best_maxw) {
            memcpy(Pbest, P, sizeof(int32_t) * (size_t)n);
            best_cut = cut; best_maxw = maxw; noimp = 0;
        }
        if (kind_count) kind_count[kind]++;
        if (it - 1 < trace_cap) {
            if (tr_kind) tr_kind[it - 1] = kind;
            if (tr_nx) tr_nx[it - 1] = nx;
            if (tr_nm) tr_nm[it - 1] = nm;
            if (tr_cut) tr_cut[it - 1] = cut;
            if (tr_maxw) tr_maxw[it - 1] = maxw;
        }
    }
    memcpy(P, Pbest, sizeof(int32_t) * (size_t)n);
    if (cut_out) *cut_out = best_cut;
    if (maxw_out) *maxw_out = best_maxw;
    if (iters_out) *iters_out = it;
    free(Pbest); free(Pd); free(dest); free(F); free(F2); free(inX); free(inM); free(locked); free(pw);
    return best_bal ? 0 : 1;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1: coarsening (heavy-edge matching) and Alg. 2 contraction   */
/* ------------------------------------------------------------------ */

/*
 * Heavy-edge matching (Sec. 3.1; the paper defers details to its earlier
 * coarsening work).  Reading, deterministic handshake rounds r = 0..R-1:
 * every unmatched v proposes the unmatched neighbour u maximising
 * (w_uv, then smaller h(r,u), then smaller u), h(r,u) = splitmix64(seed ^
 * (0xD1B54A32D192ED03 (64 level + r + 1)) ^ u); v and u match when they
 * propose each other.  Stops after the first round that adds no match.
 * mate[v] = partner or -1.  Returns the number of matched vertices.
 */
int64_t or_hem(const or_graph *g, uint64_t seed, int32_t level, int32_t rounds, int32_t *mate)
{
    int64_t n = g->n, matched = 0;
    int32_t *prop = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) mate[v] = -1;
    for (int32_t r = 0; r < rounds; ++r) {
        uint64_t salt = 0xD1B54A32D192ED03ULL * (uint64_t)(64 * (int64_t)level + r + 1);
        for (int64_t v = 0; v < n; ++v) {
            prop[v] = -1;
            if (mate[v] >= 0) continue;
            int64_t bw = 0; uint64_t bh = 0; int32_t bu = -1;
            for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; ++j) {
                int32_t u = g->adjncy[j];
                if (mate[u] >= 0) continue;
                int64_t w = ew(g, j);
                uint64_t h = or_splitmix64(seed ^ salt ^ (uint64_t)u);
                if (bu < 0 || w > bw || (w == bw && (h < bh || (h == bh && u < bu)))) { bw = w; bh = h; bu = u; }
            }
            prop[v] = bu;
        }
        int64_t added = 0;
        for (int64_t v = 0; v < n; ++v) {
            int32_t u = prop[v];
            if (u >= 0 && prop[u] == v) { mate[v] = u; ++added; }
        }
        matched += added;
        if (added == 0) break;
    }
    free(prop);
    return matched;
}

/*
 * Two-hop matching (Sec. 3.1; details are in the paper's references, not in
 * the paper).  Readings, all deterministic:
 *  - with OR_TWO_HOP set, it runs after heavy-edge matching, stage by stage (leaves, twins,
 *    relatives), each stage only while more than 25% of the vertices are
 *    unmatched (4 u > n);
 *  - leaves: unmatched vertices of degree 1, grouped by their neighbour;
 *  - twins: unmatched vertices grouped by their neighbourhood, identified by
 *    the order-free hash  splitmix64(deg ^ TWIN_DEG) + sum_u splitmix64(u ^
 *    TWIN_SALT)  (mod 2^64; the all-ones value is mapped to all-ones - 1),
 *    degree 0 included (isolated vertices are twins of each other);
 *  - relatives: unmatched vertices grouped by their matchmaker, the
 *    lowest-id neighbour that is matched when the stage starts and has
 *    degree <= OR_MATCHMAKER_MAX_DEG ("very high degree" vertices do not
 *    act as matchmakers);
 *  - inside a group, vertices are paired in ascending id: the 1st with the
 *    2nd, the 3rd with the 4th, ...; an odd last one stays unmatched.
 * added[s] (optional) receives the vertices matched by stage s.
 */
#define OR_MATCHMAKER_MAX_DEG 1024
#define OR_TWIN_SALT 0x2545F4914F6CDD1DULL
#define OR_TWIN_DEG 0x9FB21C651E98DF25ULL

typedef struct { uint64_t key; int32_t v; } or_pk;

static int pk_cmp(const void *a, const void *b)
{
    const or_pk *x = (const or_pk *)a, *y = (const or_pk *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

static int64_t pair_groups(or_pk *c, int64_t nc, int32_t *mate)
{
    qsort(c, (size_t)nc, sizeof(or_pk), pk_cmp);
    int64_t added = 0;
    for (int64_t s = 0; s < nc;) {
        int64_t e = s;
        while (e < nc && c[e].key == c[s].key) ++e;
        for (int64_t i = s; i + 1 < e; i += 2) {
            mate[c[i].v] = c[i + 1].v;
            mate[c[i + 1].v] = c[i].v;
            added += 2;
        }
        s = e;
    }
    return added;
}

uint64_t or_twin_key(const or_graph *g, int32_t v)
{
    int64_t deg = g->xadj[v + 1] - g->xadj[v];
    uint64_t h = or_splitmix64((uint64_t)deg ^ OR_TWIN_DEG);
    for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; ++j) h += or_splitmix64((uint64_t)(uint32_t)g->adjncy[j] ^ OR_TWIN_SALT);
    return h == ~0ULL ? ~0ULL - 1 : h;
}

int64_t or_two_hop(const or_graph *g, int32_t *mate, int64_t *added)
{
    int64_t n = g->n, total = 0;
    or_pk *c = (or_pk *)malloc(sizeof(or_pk) * (size_t)(n > 0 ? n : 1));
    for (int s = 0; s < 3; ++s) {
        if (added) added[s] = 0;
        int64_t un = 0;
        for (int64_t v = 0; v < n; ++v) un += mate[v] < 0;
        if (4 * un <= n) break;
        int64_t nc = 0;
        for (int64_t v = 0; v < n; ++v) {
            if (mate[v] >= 0) continue;
            int64_t deg = g->xadj[v + 1] - g->xadj[v];
            if (s == 0) {
                if (deg != 1) continue;
                c[nc].key = (uint64_t)(uint32_t)g->adjncy[g->xadj[v]];
            } else if (s == 1) {
                c[nc].key = or_twin_key(g, (int32_t)v);
            } else {
                int32_t mm = -1;
                for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; ++j) {
                    int32_t u = g->adjncy[j];
                    if (mate[u] >= 0 && g->xadj[u + 1] - g->xadj[u] <= OR_MATCHMAKER_MAX_DEG && (mm < 0 || u < mm)) mm = u;
                }
                if (mm < 0) continue;
                c[nc].key = (uint64_t)(uint32_t)mm;
            }
            c[nc].v = (int32_t)v;
            ++nc;
        }
        int64_t a = pair_groups(c, nc, mate);
        if (added) added[s] = a;
        total += a;
    }
    free(c);
    return total;
}

/* Coarse mapping C (input of Alg. 2): each matched pair and each unmatched
 * vertex becomes one coarse vertex, numbered in the order of the smaller
 * fine id of the pair.  Returns n_c. */
int32_t or_coarse_map(int32_t n, const int32_t *mate, int32_t *cmap)
{
    int32_t nc = 0;
    for (int64_t v = 0; v < n; ++v)
        if (mate[v] < 0 || v < mate[v]) cmap[v] = nc++;
    for (int64_t v = 0; v < n; ++v)
        if (mate[v] >= 0 && mate[v] < v) cmap[v] = cmap[mate[v]];
    return nc;
}

/*
 * Edge contraction (Alg. 2): the coarse graph's edges are the fine edges
 * mapped through C with parallel edges merged (weights summed).  Reading:
 * self-loops are dropped (Sec. 2.1 forbids them) and each coarse row lists
 * its neighbours in ascending id (Alg. 2's hash order is racy).  Coarse
 * vertex weights are sums.  xadj_c (nc+1) and vwgt_c (nc) are caller-owned;
 * *adj_out and *ew_out are malloc'ed here (free with or_free).
 */
int or_contract(const or_graph *g, const int32_t *cmap, int32_t nc, int64_t *xadj_c, int32_t *vwgt_c,
                int32_t **adj_out, int32_t **ew_out)
{
    int64_t n = g->n;
    /* members of each coarse vertex */
    int64_t *mstart = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) mstart[cmap[v] + 1]++;
    for (int64_t c = 0; c < nc; ++c) mstart[c + 1] += mstart[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    for (int64_t c = 0; c < nc; ++c) fill[c] = mstart[c];
    for (int64_t v = 0; v < n; ++v) mem[fill[cmap[v]]++] = (int32_t)v;
    free(fill);
    /* dense accumulator over coarse ids */
    int64_t *acc = (int64_t *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int64_t));
    int32_t *keys = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    int64_t cap = g->xadj[n] > 0 ? g->xadj[n] : 1;
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *w = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    xadj_c[0] = 0;
    for (int64_t c = 0; c < nc; ++c) {
        int64_t cw = 0; int32_t nk = 0;
        for (int64_t i = mstart[c]; i < mstart[c + 1]; ++i) {
            int64_t v = mem[i];
            cw += vw(g, v);
            for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; ++j) {
                int32_t cu = cmap[g->adjncy[j]];
                if (cu == c) continue;
                if (acc[cu] == 0) keys[nk++] = cu;
                acc[cu] += ew(g, j);
            }
        }
        /* ascending neighbour ids: insertion sort of the (few) keys */
        for (int32_t a = 1; a < nk; ++a) {
            int32_t x = keys[a]; int32_t b = a - 1;
            while (b >= 0 && keys[b] > x) { keys[b + 1] = keys[b]; --b; }
            keys[b + 1] = x;
        }
        int64_t base = xadj_c[c];
        for (int32_t a = 0; a < nk; ++a) {
            adj[base + a] = keys[a]; w[base + a] = (int32_t)acc[keys[a]]; acc[keys[a]] = 0;
        }
        xadj_c[c + 1] = base + nk;
        vwgt_c[c] = (int32_t)cw;
    }
    free(mstart); free(mem); free(acc); free(keys);
    *adj_out = adj; *ew_out = w;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Initial partition of the coarsest graph (Alg. 1 InitialPartition)   */
/* ------------------------------------------------------------------ */

/*
 * The paper calls Metis here (Sec. 3); this build uses a greedy graph-growing
 * partition instead.  Definition: order the vertices by (lowest vertex id of
 * their connected component, hop distance from that vertex, vertex id) —
 * breadth-first levels grown from the smallest id of each component — and
 * cut that sequence into k consecutive pieces by weight:
 * P(v) = floor(k S(v) / W), S(v) = weight of the vertices before v.
 */
typedef struct { int64_t root, dist; int32_t v; } or_ikey;

static int ikey_cmp(const void *a, const void *b)
{
    const or_ikey *x = (const or_ikey *)a, *y = (const or_ikey *)b;
    if (x->root != y->root) return x->root < y->root ? -1 : 1;
    if (x->dist != y->dist) return x->dist < y->dist ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

void or_initial_partition(const or_graph *g, int32_t k, int32_t *part)
{
    int64_t n = g->n;
    if (n == 0) return;
    int64_t *root = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) root[v] = -1;
    for (int64_t s = 0; s < n; ++s) {
        if (root[s] >= 0) continue;
        int64_t head = 0, tail = 0;
        root[s] = s; dist[s] = 0; queue[tail++] = (int32_t)s;
        while (head < tail) {
            int32_t v = queue[head++];
            for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; ++j) {
                int32_t u = g->adjncy[j];
                if (root[u] < 0) { root[u] = s; dist[u] = dist[v] + 1; queue[tail++] = u; }
            }
        }
    }
    or_ikey *ord = (or_ikey *)malloc(sizeof(or_ikey) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) { ord[v].root = root[v]; ord[v].dist = dist[v]; ord[v].v = (int32_t)v; }
    qsort(ord, (size_t)n, sizeof(or_ikey), ikey_cmp);
    int64_t W = 0;
    for (int64_t v = 0; v < n; ++v) W += vw(g, v);
    int64_t S = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t v = ord[i].v;
        part[v] = (int32_t)(((int64_t)k * S) / W);
        S += vw(g, v);
    }
    free(root); free(dist); free(queue); free(ord);
}

/* ------------------------------------------------------------------ */
/* Alg. 1: the multilevel template                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t levels;
    int32_t n[64];
    int64_t *xadj[64];
    int32_t *adj[64], *vwgt[64], *adjwgt[64];
    int32_t *cmap[64];   /* cmap[i]: level i -> level i+1 (NULL for the last) */
    int owns[64];        /* level 0 borrows the caller's arrays */
} or_hier;

static or_graph hier_graph(const or_hier *h, int32_t i)
{
    or_graph g = { h->n[i], h->xadj[i], h->adj[i], h->vwgt[i], h->adjwgt[i] };
    return g;
}

int32_t or_coarsen_target(int32_t k, const or_opts *o)
{
    if (o->coarsen_target > 0) return o->coarsen_target;
    return 8 * k > 256 ? 8 * k : 256;
}

/*
 * MLCoarsen (Alg. 1): repeat matching (heavy-edge, then two-hop with
 * OR_TWO_HOP) + contraction while the current graph
 * has more than T vertices (T = max(8k, 256), reading of Sec. 3's "between 4k
 * and 8k") and fewer than max_levels levels exist.  A level that would keep
 * more than 95% of the vertices is not added (coarsening stalled; reading).
 */
or_hier *or_coarsen(const or_graph *g, int32_t k, uint64_t seed, const or_opts *o)
{
    or_hier *h = (or_hier *)calloc(1, sizeof(or_hier));
    int32_t T = or_coarsen_target(k, o);
    h->levels = 1;
    h->n[0] = g->n; h->xadj[0] = (int64_t *)g->xadj; h->adj[0] = (int32_t *)g->adjncy;
    /* level 0 weights materialised when NULL so coarse sums are uniform */
    h->vwgt[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n > 0 ? g->n : 1));
    for (int64_t v = 0; v < g->n; ++v) h->vwgt[0][v] = (int32_t)vw(g, v);
    int64_t nnz = g->xadj[g->n];
    h->adjwgt[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t j = 0; j < nnz; ++j) h->adjwgt[0][j] = (int32_t)ew(g, j);
    h->owns[0] = 0;
    while (h->n[h->levels - 1] > T && h->levels < o->max_levels) {
        int32_t i = h->levels - 1;
        or_graph gi = hier_graph(h, i);
        int32_t *mate = (int32_t *)malloc(sizeof(int32_t) * (size_t)(gi.n > 0 ? gi.n : 1));
        int32_t *cmap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(gi.n > 0 ? gi.n : 1));
        or_hem(&gi, seed, i, o->hem_rounds, mate);
        if (o->flags & OR_TWO_HOP) or_two_hop(&gi, mate, NULL);
        int32_t nc = or_coarse_map(gi.n, mate, cmap);
        free(mate);
        if ((int64_t)100 * nc > (int64_t)95 * gi.n) { free(cmap); break; }
        int64_t *xc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
        int32_t *vc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
        int32_t *ac = NULL, *wc = NULL;
        or_contract(&gi, cmap, nc, xc, vc, &ac, &wc);
        h->cmap[i] = cmap;
        h->n[i + 1] = nc; h->xadj[i + 1] = xc; h->adj[i + 1] = ac; h->vwgt[i + 1] = vc; h->adjwgt[i + 1] = wc;
        h->owns[i + 1] = 1;
        h->levels++;
    }
    return h;
}

void or_hier_free(or_hier *h)
{
    if (!h) return;
    for (int32_t i = 0; i < h->levels; ++i) {
        if (h->owns[i]) { free(h->xadj[i]); free(h->adj[i]); }
        free(h->vwgt[i]); free(h->adjwgt[i]); free(h->cmap[i]);
    }
    free(h);
}

int32_t or_hier_levels(const or_hier *h) { return h->levels; }

void or_hier_get(const or_hier *h, int32_t i, int32_t *n, int64_t **xadj, int32_t **adj, int32_t **vwgt,
                 int32_t **adjwgt, int32_t **cmap)
{
    *n = h->n[i]; *xadj = h->xadj[i]; *adj = h->adj[i]; *vwgt = h->vwgt[i]; *adjwgt = h->adjwgt[i];
    *cmap = h->cmap[i];
}

/* Seed of Jetrw's hash on level i: splitmix64(seed ^ 0xA0761D6478BD642F (i+1)) */
uint64_t or_level_seed(uint64_t seed, int32_t level)
{
    return or_splitmix64(seed ^ (0xA0761D6478BD642FULL * (uint64_t)(level + 1)));
}

/*
 * Alg. 1 after MLCoarsen: InitialPartition on the coarsest level, then
 * RefinePartition there and, for each finer level, ProjectPartition
 * (P_i[v] = P_{i+1}[C_i[v]]) followed by RefinePartition.  c = c_fine on
 * level 0, c_coarse elsewhere (Sec. 4.1.2).  Returns the final refine status.
 */
int or_uncoarsen(const or_hier *h, int32_t k, double eps, uint64_t seed, const or_opts *o,
                 int32_t *part_out, int64_t *cut_out, or_stats *st)
{
    int32_t l = h->levels - 1;
    int32_t *P = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->n[l] > 0 ? h->n[l] : 1));
    double t0 = or_now();
    or_graph gl = hier_graph(h, l);
    or_initial_partition(&gl, k, P);
    double t1 = or_now();
    int status = 0;
    int64_t cut = 0, maxw = 0;
    for (int32_t i = l; i >= 0; --i) {
        or_graph gi = hier_graph(h, i);
        if (i < l) {
            int32_t *Pi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(gi.n > 0 ? gi.n : 1));
            for (int64_t v = 0; v < gi.n; ++v) Pi[v] = P[h->cmap[i][v]];
            free(P); P = Pi;
        }
        int32_t iters = 0, kc[3];
        double ts = or_now();
        status = or_refine(&gi, k, eps, i == 0 ? o->c_fine_q16 : o->c_coarse_q16, or_level_seed(seed, i), o,
                           P, &cut, &maxw, 0, NULL, NULL, NULL, NULL, NULL, &iters, kc);
        if (st) {
            st->it_lp[i] = kc[0]; st->it_rw[i] = kc[1]; st->it_rs[i] = kc[2];
            st->cut_level[i] = cut;
            st->edge_iters += (int64_t)iters * (gi.xadj[gi.n] / 2);
            if (i == 0) { st->fin_edge_iters = (int64_t)iters * (gi.xadj[gi.n] / 2); st->sec_refine_finest = or_now() - ts; }
        }
    }
    double t2 = or_now();
    memcpy(part_out, P, sizeof(int32_t) * (size_t)h->n[0]);
    free(P);
    if (cut_out) *cut_out = cut;
    if (st) {
        st->levels = h->levels;
        for (int32_t i = 0; i < h->levels; ++i) { st->n[i] = h->n[i]; st->m[i] = h->xadj[i][h->n[i]] / 2; }
        st->cut = cut; st->maxw = maxw;
        st->sec_init = t1 - t0; st->sec_refine = t2 - t1;
    }
    return status;
}

/* jet_partition's definition: Alg. 1 end to end. */
int or_partition(const or_graph *g, int32_t k, double eps, uint64_t seed, const or_opts *o,
                 int32_t *part_out, int64_t *cut_out, or_stats *st)
{
    if (st) memset(st, 0, sizeof(*st));
    double t0 = or_now();
    or_hier *h = or_coarsen(g, k, seed, o);
    double t1 = or_now();
    int status = or_uncoarsen(h, k, eps, seed, o, part_out, cut_out, st);
    if (st) st->sec_coarsen = t1 - t0;
    or_hier_free(h);
    return status;
}
