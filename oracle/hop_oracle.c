/*
 * HOP oracle: a plain, slow, obviously correct CPU implementation in fp64.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code,
 * header, table or helper with the CUDA path and must never be used by it.
 *
 * What it computes follows the HOP method as restated in Parallel HOP
 * (Skory et al., arXiv:1001.3411), Section 2, with the readings listed
 * beside each function where the paper is silent:
 *
 *   C1 knn         exact Ndens nearest neighbours, self included (Sec. 2,
 *                  first paragraph), periodic minimum image, order (d^2, j).
 *   C2 density     SPH cubic-spline (M4) density over the Ndens list,
 *                  normalised to the mean particle density of the box (Sec. 2).
 *   C3 link        hop to the densest of the first Nhop list entries, which
 *                  may be the particle itself (Sec. 2, second paragraph).
 *   C4 chains      follow hops uphill to a particle that is its own densest
 *                  neighbour (Sec. 2).
 *   C5 boundaries  max over particle pairs of the summed density, per chain
 *                  pair, over the first Nmerge entries (Sec. 2, merging step 3;
 *                  links may be one-directional).
 *   C6 merge       proto-halos (peak >= delta_peak) merge when their boundary
 *                  is >= delta_saddle (step 4); sub-peak chains join the
 *                  proto-halo reached along the densest propagated boundary
 *                  (step 5, Fig. 1).
 *   C7 labels      particles below delta_outer are in no halo (step 1);
 *                  groups are numbered by (peak density desc, peak index asc).
 *   C8 halo stats  mass, centre of mass and maximum radius of every halo
 *                  (Sec. 3, last paragraph of the merging description).
 *   C9 subhalos    ADAPTAHOP's extension (Sec. 6): symmetric boundaries
 *                  only, links below a threshold delta_s destroyed, one
 *                  labelling per delta_s, Poisson significance cut.
 *
 * Arithmetic: positions are taken as doubles (fp32 inputs promote exactly);
 * distances, kernel sums and boundary sums are fp64.  Densities handed in
 * from elsewhere (the "fed the same arrays" protocol) are doubles holding
 * the exact fp32 values, so every comparison is exact.
 *
 * Parallelism: OpenMP over independent particles only (C1-C3).  Everything
 * order-dependent (chains, the boundary table, the merge) is sequential.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ECYCLE 3
#define ORC_ECAP 4

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Periodic minimum-image component: the image of dx closest to zero. */
static double min_image(double dx, double box)
{
    if (dx > 0.5 * box) return dx - box;
    if (dx < -0.5 * box) return dx + box;
    return dx;
}

/* (d2a, ja) strictly before (d2b, jb) in the list order of C1. */
static int knn_before(double d2a, int32_t ja, double d2b, int32_t jb)
{
    return d2a < d2b || (d2a == d2b && ja < jb);
}

/*
 * C1.  For each query i (queries[q], or q when queries is NULL) the k
 * particles j (the query itself included, at d^2 = 0) with the smallest
 * periodic d^2(i, j), listed in ascending (d^2, j).  Brute force over all n.
 * nbr and d2 are nq x k, row-major.
 */
int orc_knn(const double *pos, int64_t n, double box, int32_t k,
            const int64_t *queries, int64_t nq, int32_t *nbr, double *d2)
{
    if (!pos || n <= 0 || k <= 0 || k > n || !nbr || !d2 || !(box > 0)) return ORC_EINVAL;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = queries ? queries[q] : q;
        if (i < 0 || i >= n) { bad = 1; continue; }
        double *bd = d2 + q * k;
        int32_t *bj = nbr + q * k;
        for (int32_t t = 0; t < k; ++t) { bd[t] = INFINITY; bj[t] = INT32_MAX; }
        const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        for (int64_t j = 0; j < n; ++j) {
            double dx = min_image(pos[3 * j] - xi, box);
            double dy = min_image(pos[3 * j + 1] - yi, box);
            double dz = min_image(pos[3 * j + 2] - zi, box);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (!knn_before(r2, (int32_t)j, bd[k - 1], bj[k - 1])) continue;
            int32_t t = k - 1;
            while (t > 0 && knn_before(r2, (int32_t)j, bd[t - 1], bj[t - 1])) {
                bd[t] = bd[t - 1];
                bj[t] = bj[t - 1];
                --t;
            }
            bd[t] = r2;
            bj[t] = (int32_t)j;
        }
    }
    return bad ? ORC_EINVAL : ORC_OK;
}

/*
 * The M4 cubic spline of Monaghan & Lattanzio (1985) in 3D, with compact
 * support 2h:  W(r, h) = w(r/h) / (pi h^3),
 *   w(q) = 1 - 1.5 q^2 + 0.75 q^3   for 0 <= q < 1,
 *        = 0.25 (2 - q)^3           for 1 <= q < 2,
 *        = 0                        otherwise.
 */
static double m4_w(double q)
{
    if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    if (q < 2.0) { double t = 2.0 - q; return 0.25 * t * t * t; }
    return 0.0;
}

/*
 * C2.  h_i = r_k / 2, where r_k is the distance to the last (k-th) list
 * entry, so the support 2h reaches exactly the farthest neighbour.
 * delta_i = (box^3 / n_total) * sum_{j in list} W(r_ij, h_i): the kernel
 * density of equal-mass particles divided by the box's mean particle
 * density.  When all k entries sit at distance 0 the density is +inf.
 */
int orc_density(const double *d2, int64_t nq, int32_t k, int64_t n_total,
                double box, double *dens)
{
    if (!d2 || !dens || k <= 0 || n_total <= 0) return ORC_EINVAL;
    const double norm = box * box * box / (double)n_total;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nq; ++q) {
        const double *row = d2 + q * k;
        double h = 0.5 * sqrt(row[k - 1]);
        if (!(h > 0)) { dens[q] = INFINITY; continue; }
        double s = 0.0;
        for (int32_t t = 0; t < k; ++t) s += m4_w(sqrt(row[t]) / h);
        dens[q] = norm * s / (M_PI * h * h * h);
    }
    return ORC_OK;
}

/* Key order of C3: higher density first, then the smaller particle index. */
static int key_greater(const double *dens, int32_t a, int32_t b)
{
    return dens[a] > dens[b] || (dens[a] == dens[b] && a < b);
}

/*
 * C3 + C4.  hop_i = the densest of the first n_hop entries of i's list
 * (ties to the smaller index); chain_i = the particle reached by following
 * hops until a particle is its own hop.  Returns ORC_ECYCLE if following
 * ever revisits a particle without reaching such a root.
 */
int orc_link(const double *dens, const int32_t *nbr, int32_t ld, int64_t n,
             int32_t n_hop, int32_t *hop, int32_t *chain)
{
    if (!dens || !nbr || !hop || !chain || n_hop <= 0 || ld < n_hop) return ORC_EINVAL;
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const int32_t *row = nbr + i * (int64_t)ld;
        int32_t best = row[0];
        if (best < 0 || best >= n) { bad = 1; continue; }
        for (int32_t t = 1; t < n_hop; ++t) {
            int32_t j = row[t];
            if (j < 0 || j >= n) { bad = 1; break; }
            if (key_greater(dens, j, best)) best = j;
        }
        hop[i] = best;
    }
    if (bad) return ORC_EINVAL;
    /* Follow each path to its root; every particle on a resolved path is
     * labelled with that root (plain memoisation of the same walk). */
    for (int64_t i = 0; i < n; ++i) chain[i] = -1;
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!path) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; ++i) {
        if (chain[i] >= 0) continue;
        int64_t len = 0;
        int32_t p = (int32_t)i;
        int32_t root = -1;
        for (;;) {
            if (chain[p] >= 0) { root = chain[p]; break; }
            if (hop[p] == p) { root = p; break; }
            if (len >= n) { free(path); return ORC_ECYCLE; }
            path[len++] = p;
            p = hop[p];
        }
        chain[p] = root;
        for (int64_t t = 0; t < len; ++t) chain[path[t]] = root;
    }
    free(path);
    return ORC_OK;
}

typedef struct { int32_t lo, hi; double s; } orc_link_t;

static int link_cmp(const void *pa, const void *pb)
{
    const orc_link_t *a = (const orc_link_t *)pa, *b = (const orc_link_t *)pb;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    if (a->s != b->s) return a->s > b->s ? -1 : 1; /* largest first */
    return 0;
}

/*
 * C5.  For every particle i with dens_i >= d_outer and every entry j of the
 * first n_merge entries of its list with j != i, dens_j >= d_outer and
 * chain_i != chain_j: the pair {chain_i, chain_j} records
 * s = dens_i + dens_j (twice the average density; the sum of two fp32 values
 * is exact in fp64).  The table keeps the maximum per pair.  Output is one
 * entry per pair, ordered by (lo, hi) with lo < hi the two chain labels.
 * *n_out is always set to the number of pairs; with lo/hi/s NULL the call
 * only reports it, and with cap too small it returns ORC_ECAP.
 */
int orc_boundaries(const int32_t *chain, const double *dens, const int32_t *nbr,
                   int32_t ld, int64_t n, int32_t n_merge, double d_outer,
                   int32_t *lo, int32_t *hi, double *s, int64_t cap, int64_t *n_out)
{
    if (!chain || !dens || !nbr || !n_out || n_merge <= 0 || ld < n_merge) return ORC_EINVAL;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(dens[i] >= d_outer)) continue;
        for (int32_t t = 0; t < n_merge; ++t) {
            int32_t j = nbr[i * (int64_t)ld + t];
            if (j < 0 || j >= n) return ORC_EINVAL;
            if (j == i || !(dens[j] >= d_outer) || chain[i] == chain[j]) continue;
            ++m;
        }
    }
    orc_link_t *raw = (orc_link_t *)malloc(sizeof(orc_link_t) * (size_t)(m ? m : 1));
    if (!raw) return ORC_ENOMEM;
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(dens[i] >= d_outer)) continue;
        for (int32_t t = 0; t < n_merge; ++t) {
            int32_t j = nbr[i * (int64_t)ld + t];
            if (j == i || !(dens[j] >= d_outer) || chain[i] == chain[j]) continue;
            int32_t a = chain[i], b = chain[j];
            raw[w].lo = a < b ? a : b;
            raw[w].hi = a < b ? b : a;
            raw[w].s = dens[i] + dens[j];
            ++w;
        }
    }
    qsort(raw, (size_t)w, sizeof(orc_link_t), link_cmp);
    int64_t u = 0;
    for (int64_t t = 0; t < w; ++t)
        if (t == 0 || raw[t].lo != raw[t - 1].lo || raw[t].hi != raw[t - 1].hi) ++u;
    *n_out = u;
    if (!lo || !hi || !s) { free(raw); return ORC_OK; } /* size query only */
    if (u > cap) { free(raw); return ORC_ECAP; }
    int64_t e = 0;
    for (int64_t t = 0; t < w; ++t) {
        if (t == 0 || raw[t].lo != raw[t - 1].lo || raw[t].hi != raw[t - 1].hi) {
            lo[e] = raw[t].lo; hi[e] = raw[t].hi; s[e] = raw[t].s; ++e;
        }
    }
    free(raw);
    return ORC_OK;
}

/* Union-find root with path halving. */
static int32_t uf_find(int32_t *parent, int32_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

typedef struct { double s; int32_t lo, hi; } orc_edge_t;

/* Strict merge order of C6: boundary descending, then lo, then hi ascending. */
static int edge_cmp(const void *pa, const void *pb)
{
    const orc_edge_t *a = (const orc_edge_t *)pa, *b = (const orc_edge_t *)pb;
    if (a->s != b->s) return a->s > b->s ? -1 : 1;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    return 0;
}

typedef struct { double d; int32_t idx; int32_t set; } orc_peak_t;

static int peak_cmp(const void *pa, const void *pb)
{
    const orc_peak_t *a = (const orc_peak_t *)pa, *b = (const orc_peak_t *)pb;
    if (a->d != b->d) return a->d > b->d ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

/*
 * C6 + C7.  Chains are the distinct values of chain[].  A chain's peak is
 * its member with the greatest key (density, then smaller index); the chain
 * is a proto-halo when the peak density is >= d_peak.
 *   (i)   every proto-halo starts as its own owned set;
 *   (ii)  proto-halo pairs whose boundary s >= 2 d_saddle are united
 *         (transitively) -- "always merge" of Sec. 2 step 4;
 *   (iii) all boundaries are then taken in strict order (s desc, lo asc,
 *         hi asc); an edge whose ends are in the same set, or in two owned
 *         sets, is skipped; otherwise the two sets unite and the result is
 *         owned if either was.  A sub-peak chain thus joins the proto-halo
 *         reached along its densest propagated boundary, and proto-halos
 *         unite only through direct boundaries >= 2 d_saddle;
 *   (iv)  a set that never becomes owned is no halo.
 * group[i] = -1 when dens_i < d_outer or i's chain is in no owned set;
 * otherwise the rank of its set when sets are ordered by their peak
 * (density desc, index asc).  *n_groups = number of owned sets.
 */
int orc_merge(const int32_t *chain, const double *dens, int64_t n,
              const int32_t *lo, const int32_t *hi, const double *s, int64_t ne,
              double d_outer, double d_saddle, double d_peak,
              int32_t *group, int64_t *n_groups)
{
    if (!chain || !dens || !group || !n_groups || n <= 0) return ORC_EINVAL;
    int rc = ORC_ENOMEM;
    int32_t *peak = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    unsigned char *owned = (unsigned char *)calloc((size_t)n, 1);
    orc_edge_t *edges = (orc_edge_t *)malloc(sizeof(orc_edge_t) * (size_t)(ne ? ne : 1));
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    orc_peak_t *pk = NULL;
    if (!peak || !parent || !owned || !edges || !rank) goto done;
    rc = ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i) { peak[i] = -1; parent[i] = (int32_t)i; rank[i] = -1; }
    /* Peak of each chain: its member with the greatest key. */
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = chain[i];
        if (c < 0 || c >= n) goto done;
        if (peak[c] < 0 || key_greater(dens, (int32_t)i, peak[c])) peak[c] = (int32_t)i;
    }
    for (int64_t c = 0; c < n; ++c)
        if (peak[c] >= 0 && dens[peak[c]] >= d_peak) owned[c] = 1;
    for (int64_t e = 0; e < ne; ++e)
        if (lo[e] < 0 || lo[e] >= n || hi[e] < 0 || hi[e] >= n ||
            peak[lo[e]] < 0 || peak[hi[e]] < 0) goto done;
    /* (ii) */
    for (int64_t e = 0; e < ne; ++e) {
        if (owned[lo[e]] && owned[hi[e]] && s[e] >= 2.0 * d_saddle) {
            int32_t a = uf_find(parent, lo[e]), b = uf_find(parent, hi[e]);
            if (a != b) parent[a] = b;
        }
    }
    /* A set is owned when it holds a proto-halo. */
    for (int64_t c = 0; c < n; ++c)
        if (owned[c]) owned[uf_find(parent, (int32_t)c)] = 1;
    /* (iii) */
    for (int64_t e = 0; e < ne; ++e) { edges[e].s = s[e]; edges[e].lo = lo[e]; edges[e].hi = hi[e]; }
    qsort(edges, (size_t)ne, sizeof(orc_edge_t), edge_cmp);
    for (int64_t e = 0; e < ne; ++e) {
        int32_t a = uf_find(parent, edges[e].lo), b = uf_find(parent, edges[e].hi);
        if (a == b || (owned[a] && owned[b])) continue;
        parent[a] = b;
        owned[b] = (unsigned char)(owned[a] | owned[b]);
    }
    /* (iv) + C7: a set's peak is the greatest chain peak among its chains;
     * owned sets are numbered by that peak (density desc, index asc). */
    int64_t ng = 0;
    for (int64_t c = 0; c < n; ++c) rank[c] = -1; /* rank[] holds set peaks here */
    for (int64_t c = 0; c < n; ++c) {
        if (peak[c] < 0) continue;
        int32_t r = uf_find(parent, (int32_t)c);
        if (!owned[r]) continue;
        if (rank[r] < 0) ++ng;
        if (rank[r] < 0 || key_greater(dens, peak[c], rank[r])) rank[r] = peak[c];
    }
    pk = (orc_peak_t *)malloc(sizeof(orc_peak_t) * (size_t)(ng ? ng : 1));
    if (!pk) { rc = ORC_ENOMEM; goto done; }
    int64_t g = 0;
    for (int64_t c = 0; c < n; ++c) {
        if (rank[c] < 0) continue;
        pk[g].d = dens[rank[c]]; pk[g].idx = rank[c]; pk[g].set = (int32_t)c; ++g;
    }
    qsort(pk, (size_t)ng, sizeof(orc_peak_t), peak_cmp);
    for (int64_t t = 0; t < ng; ++t) rank[pk[t].set] = (int32_t)t;
    for (int64_t i = 0; i < n; ++i) {
        int32_t r = uf_find(parent, chain[i]);
        group[i] = (dens[i] >= d_outer && owned[r]) ? rank[r] : -1;
    }
    *n_groups = ng;
    rc = ORC_OK;
done:
    free(peak); free(parent); free(owned); free(edges); free(rank); free(pk);
    return rc;
}

/*
 * C8.  The statistical properties the paper computes for every halo once
 * the halos are known: dark matter mass, centre of mass and maximum radius.
 * Readings: particle masses are equal, so a halo's mass is its member
 * count.  In the periodic box the centre of mass is taken about the halo's
 * peak particle (its member with the greatest key: density, then smaller
 * index): the members' minimum-image offsets from the peak are averaged and
 * added to the peak's position, then wrapped into [0, box).  The maximum
 * radius is the largest minimum-image distance from that centre to a member.
 * Outputs for g < n_groups: count[g], peak[g], com[3g .. 3g+2], rmax[g].
 * A group id >= n_groups is an error; ids < 0 are no halo.
 */
int orc_halo_stats(const double *pos, const double *dens, const int32_t *group, int64_t n,
                   int64_t n_groups, double box, int64_t *count, int32_t *peak, double *com,
                   double *rmax)
{
    if (!pos || !dens || !group || n < 0 || n_groups < 0 || !(box > 0)) return ORC_EINVAL;
    if (n_groups == 0) return ORC_OK;
    if (!count || !peak || !com || !rmax) return ORC_EINVAL;
    double *sum = (double *)calloc((size_t)n_groups * 3, sizeof(double));
    if (!sum) return ORC_ENOMEM;
    for (int64_t g = 0; g < n_groups; ++g) { count[g] = 0; peak[g] = -1; rmax[g] = 0.0; }
    for (int64_t i = 0; i < n; ++i) {
        const int32_t g = group[i];
        if (g < 0) continue;
        if (g >= n_groups) { free(sum); return ORC_EINVAL; }
        ++count[g];
        if (peak[g] < 0 || key_greater(dens, (int32_t)i, peak[g])) peak[g] = (int32_t)i;
    }
    for (int64_t i = 0; i < n; ++i) {
        const int32_t g = group[i];
        if (g < 0) continue;
        for (int d = 0; d < 3; ++d)
            sum[3 * g + d] += min_image(pos[3 * i + d] - pos[3 * (int64_t)peak[g] + d], box);
    }
    for (int64_t g = 0; g < n_groups; ++g) {
        for (int d = 0; d < 3; ++d) {
            double c = count[g] > 0 ? pos[3 * (int64_t)peak[g] + d] + sum[3 * g + d] / (double)count[g] : 0.0;
            if (c < 0.0) c += box;
            if (c >= box) c -= box;
            com[3 * g + d] = c;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        const int32_t g = group[i];
        if (g < 0) continue;
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double dx = min_image(pos[3 * i + d] - com[3 * g + d], box);
            r2 += dx * dx;
        }
        const double r = sqrt(r2);
        if (r > rmax[g]) rmax[g] = r;
    }
    free(sum);
    return ORC_OK;
}

/* Directed link a -> b with its summed density; ordered by (a, b, s desc). */
typedef struct { int32_t a, b; double s; } orc_dlink_t;

static int dlink_cmp(const void *pa, const void *pb)
{
    const orc_dlink_t *x = (const orc_dlink_t *)pa, *y = (const orc_dlink_t *)pb;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    if (x->s != y->s) return x->s > y->s ? -1 : 1;
    return 0;
}

/*
 * C9a.  ADAPTAHOP's symmetric boundaries (Sec. 6, subhalos).  A directed
 * link a -> b exists when some particle i of chain a with dens_i >= d_outer
 * has, among the first n_merge entries of its list, a j != i of chain
 * b != a with dens_j >= d_outer (the particle filter of C5).  A pair {a, b}
 * is a symmetric boundary only when both a -> b and b -> a exist; its value
 * s is the largest dens_i + dens_j over the links of both directions (the
 * value C5 gives the same pair).  Output as in C5: one entry per kept pair,
 * ordered by (lo, hi); *n_out is always set; with lo/hi/s NULL the call
 * only reports it, and with cap too small it returns ORC_ECAP.
 */
int orc_sym_boundaries(const int32_t *chain, const double *dens, const int32_t *nbr,
                       int32_t ld, int64_t n, int32_t n_merge, double d_outer,
                       int32_t *lo, int32_t *hi, double *s, int64_t cap, int64_t *n_out)
{
    if (!chain || !dens || !nbr || !n_out || n_merge <= 0 || ld < n_merge) return ORC_EINVAL;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(dens[i] >= d_outer)) continue;
        for (int32_t t = 0; t < n_merge; ++t) {
            const int32_t j = nbr[i * (int64_t)ld + t];
            if (j < 0 || j >= n) return ORC_EINVAL;
            if (j == i || !(dens[j] >= d_outer) || chain[i] == chain[j]) continue;
            ++m;
        }
    }
    orc_dlink_t *raw = (orc_dlink_t *)malloc(sizeof(orc_dlink_t) * (size_t)(m ? m : 1));
    if (!raw) return ORC_ENOMEM;
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(dens[i] >= d_outer)) continue;
        for (int32_t t = 0; t < n_merge; ++t) {
            const int32_t j = nbr[i * (int64_t)ld + t];
            if (j == i || !(dens[j] >= d_outer) || chain[i] == chain[j]) continue;
            raw[w].a = chain[i];
            raw[w].b = chain[j];
            raw[w].s = dens[i] + dens[j];
            ++w;
        }
    }
    qsort(raw, (size_t)w, sizeof(orc_dlink_t), dlink_cmp);
    /* keep the first (largest s) entry of every directed pair */
    int64_t d = 0;
    for (int64_t t = 0; t < w; ++t)
        if (t == 0 || raw[t].a != raw[t - 1].a || raw[t].b != raw[t - 1].b) raw[d++] = raw[t];
    /* a -> b with a < b is kept when b -> a exists (binary search) */
    int64_t u = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            *n_out = u;
            if (!lo || !hi || !s) break;
            if (u > cap) { free(raw); return ORC_ECAP; }
            u = 0;
        }
        for (int64_t t = 0; t < d; ++t) {
            if (raw[t].a > raw[t].b) continue;
            int64_t l = 0, r = d;
            while (l < r) {
                const int64_t mid = l + (r - l) / 2;
                if (raw[mid].a < raw[t].b || (raw[mid].a == raw[t].b && raw[mid].b < raw[t].a)) l = mid + 1;
                else r = mid;
            }
            if (l == d || raw[l].a != raw[t].b || raw[l].b != raw[t].a) continue;
            if (pass == 1) {
                lo[u] = raw[t].a;
                hi[u] = raw[t].b;
                s[u] = raw[t].s > raw[l].s ? raw[t].s : raw[l].s;
            }
            ++u;
        }
    }
    free(raw);
    return ORC_OK;
}

/*
 * C9b.  Subhalos at each threshold delta_s = levels[l] (Sec. 6): every
 * boundary with s < 2 delta_s (a link density below delta_s) is destroyed
 * and chains joined by the remaining boundaries merge, transitively (the
 * connected components of the chain graph).  A particle belongs to its
 * component's subhalo when dens_i >= delta_s.  A component with N >= 1 such
 * members is rejected when N < n_min or when their mean density (fp64 sum
 * in index order, divided by N) is below delta_s * (1 + f_poisson / sqrt(N)),
 * the relative Poisson noise of a count of N scaled by f_poisson.  Accepted
 * subhalos of a level are numbered by their peak member (density desc,
 * index asc).  sub[l * n + i] = that number, or -1; n_sub[l] = the number
 * accepted.  Boundary ends are chain labels in [0, n).
 */
int orc_subhalos(const int32_t *chain, const double *dens, int64_t n,
                 const int32_t *lo, const int32_t *hi, const double *s, int64_t ne,
                 const double *levels, int32_t n_levels, int64_t n_min, double f_poisson,
                 int32_t *sub, int64_t *n_sub)
{
    if (!chain || !dens || !levels || !sub || !n_sub || n <= 0 || n_levels <= 0 || n_min < 1 ||
        !(f_poisson >= 0.0))
        return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        if (chain[i] < 0 || chain[i] >= n) return ORC_EINVAL;
    for (int64_t e = 0; e < ne; ++e)
        if (lo[e] < 0 || lo[e] >= n || hi[e] < 0 || hi[e] >= n) return ORC_EINVAL;
    int rc = ORC_ENOMEM;
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *sum = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *peak = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    orc_peak_t *pk = (orc_peak_t *)malloc(sizeof(orc_peak_t) * (size_t)n);
    if (!parent || !cnt || !sum || !peak || !rank || !pk) goto done;
    for (int32_t l = 0; l < n_levels; ++l) {
        const double ds = levels[l];
        for (int64_t c = 0; c < n; ++c) { parent[c] = (int32_t)c; cnt[c] = 0; sum[c] = 0.0; peak[c] = -1; rank[c] = -1; }
        for (int64_t e = 0; e < ne; ++e) {
            if (!(s[e] >= 2.0 * ds)) continue;
            const int32_t a = uf_find(parent, lo[e]), b = uf_find(parent, hi[e]);
            if (a != b) parent[a] = b;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (!(dens[i] >= ds)) continue;
            const int32_t r = uf_find(parent, chain[i]);
            ++cnt[r];
            sum[r] += dens[i];
            if (peak[r] < 0 || key_greater(dens, (int32_t)i, peak[r])) peak[r] = (int32_t)i;
        }
        int64_t g = 0;
        for (int64_t c = 0; c < n; ++c) {
            if (cnt[c] == 0 || cnt[c] < n_min) continue;
            const double N = (double)cnt[c];
            if (!(sum[c] / N >= ds * (1.0 + f_poisson / sqrt(N)))) continue;
            pk[g].d = dens[peak[c]]; pk[g].idx = peak[c]; pk[g].set = (int32_t)c; ++g;
        }
        qsort(pk, (size_t)g, sizeof(orc_peak_t), peak_cmp);
        for (int64_t t = 0; t < g; ++t) rank[pk[t].set] = (int32_t)t;
        int32_t *out = sub + (int64_t)l * n;
        for (int64_t i = 0; i < n; ++i)
            out[i] = dens[i] >= ds ? rank[uf_find(parent, chain[i])] : -1;
        n_sub[l] = g;
    }
    rc = ORC_OK;
done:
    free(parent); free(cnt); free(sum); free(peak); free(rank); free(pk);
    return rc;
}
