/*
 * hop.h -- C ABI of the GB300 HOP halo finder (libhop.so).
 *
 * HOP (Eisenstein & Hut 1998) as restated in Parallel HOP (Skory, Turk,
 * Norman & Coil, arXiv:1001.3411, Sec. 2) assigns every particle of a
 * periodic box to a density-peak group:
 *   1. the Ndens nearest neighbours of each particle, itself included, give
 *      an SPH kernel density normalised to the mean particle density;
 *   2. each particle hops to the densest of its first Nhop neighbours
 *      (possibly itself), and hops are followed uphill to a peak (a chain);
 *   3. over the first Nmerge neighbours, the densest pair straddling two
 *      chains gives their boundary density;
 *   4. chains merge into groups under delta_outer, delta_saddle, delta_peak.
 * Sec. 4 ("Modular Portability") states the interface the calls below
 * follow: positions and box bounds in, per-particle group ids and kernel
 * densities out.
 *
 * Conventions shared by every call
 *   - Particles are indexed 0..n-1 in the caller's order.  All index arrays
 *     (neighbour lists, hops, chain labels, boundary pairs) hold these
 *     indices as uint32.  n must be < 2^31.
 *   - Positions are AoS, 3 values per particle, in [0, box).  A coordinate
 *     outside [0, box) (or NaN) makes the call fail with HOP_EINVAL.
 *   - Pointers are device pointers unless a call says otherwise; calls
 *     that also accept host memory say so and detect it themselves.
 *   - The caller owns every input and output buffer.  The context owns its
 *     scratch memory (grown on demand, kept between calls) and a stream.
 *   - All calls are enqueued on the context's stream.  A call returns after
 *     its work is enqueued, except where it must read a count back to the
 *     host (noted per call); those calls synchronise the stream.
 *   - Return codes are HOP_* below.  No C++ exception crosses the ABI.
 *     hop_last_error() describes the last failure of a context.
 */
#ifndef HOP_H_
#define HOP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HOP_OK = 0,
    HOP_EINVAL = 1,      /* bad argument: sizes, ranges, null pointers, positions   */
    HOP_ENOMEM = 2,      /* device allocation failed                                */
    HOP_ECUDA = 3,       /* a CUDA runtime call failed (message in hop_last_error)  */
    HOP_ETABLE = 4,      /* caller's edge capacity too small; *n_edges = required   */
    HOP_ETIMEOUT = 5,    /* a device loop reached its iteration limit               */
    HOP_EDEGENERATE = 6, /* more equidistant neighbours than the search buffer holds */
    HOP_ENOMODEL = 7,    /* learned radius requested but no network is loaded        */
    HOP_ESTATIC = 8      /* n exceeds the fixed scratch of hop_link_static           */
};

/* How the kNN search picks each warp's first search radius.  All three give
 * identical results: a search is certified only when at least Ndens
 * particles fall inside a radius whose ball was scanned completely, and is
 * otherwise repeated with a larger radius. */
enum {
    HOP_RADIUS_PLAIN = 0,   /* mean-density Ndens-th-neighbour distance, expanded    */
    HOP_RADIUS_COUNT = 1,   /* closed form from the 27 stencil cell counts          */
    HOP_RADIUS_LEARNED = 2  /* the loaded MLP reads the 27 log-counts (hop_mlp_*)   */
};

typedef struct hop_params {
    int32_t n_dens;       /* Ndens: list length incl. self (Sec. 2); 2..128        */
    int32_t n_hop;        /* Nhop: hop candidates, 1..n_dens                         */
    int32_t n_merge;      /* Nmerge: boundary search, 1..n_hop                      */
    float delta_outer;    /* delta_outer: no halo below it (Sec. 2, step 1)         */
    float delta_saddle;   /* delta_saddle: proto-halo merge threshold (step 4)      */
    float delta_peak;     /* delta_peak: proto-halo threshold (step 2)              */
    double box;           /* periodic box side L > 0                                */
    int32_t pos_is_f64;   /* 0: positions are float32; 1: float64 (fp64 distances)  */
    int32_t radius_mode;  /* HOP_RADIUS_*                                           */
} hop_params;

/* Fills p with the parameters the hot path is benchmarked with:
 * Ndens 64, Nhop 16, Nmerge 4, delta 80 / 200 / 240, box 1, fp32, plain.
 * (The paper's own defaults, Table 2, are Ndens = Nhop = 65, Nmerge = 4,
 * delta_saddle = 2.5 delta_outer, delta_peak = 3 delta_outer.) */
void hop_default_params(hop_params *p);

typedef struct hop_ctx hop_ctx;

/* Creates a context on CUDA device `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Returns HOP_OK and
 * *out, or an error code and *out = NULL. */
int hop_create(hop_ctx **out, int device, void *cuda_stream);
/* Frees the context's scratch memory.  Safe on NULL. */
void hop_destroy(hop_ctx *ctx);
/* Changes the stream later calls enqueue on. */
int hop_set_stream(hop_ctx *ctx, void *cuda_stream);
/* Message of the last failure on this context ("" when none).  The string
 * lives until the next call on the context. */
const char *hop_last_error(const hop_ctx *ctx);
/* Sets the queries per warp of the kNN search (1, 2, 4, 8, 16 or 32) and
 * the number of search cells per radius (1 to 4); 0 keeps the current value.
 * Results do not depend on these; only speed does. */
int hop_set_tuning(hop_ctx *ctx, int32_t queries_per_warp, int32_t cells_per_radius);

/*
 * Step 1 (Sec. 2): Ndens nearest neighbours and kernel density.
 *   pos   n x 3 float32 or float64 (params->pos_is_f64), AoS, device.
 *   nbr   n x ld_nbr uint32: row i holds the first ld_nbr entries of i's
 *         neighbour list in ascending (d^2, index) order, the particle itself
 *         included (at d^2 = 0).  n_hop <= ld_nbr <= n_dens.  May be NULL.
 *   dens  n float32: delta_i = (L^3/n) sum_{j in list} W(r_ij, h_i), W the M4
 *         cubic spline with support 2h_i = r_k (the last list entry's
 *         distance); +inf when all Ndens entries are at distance 0.
 *   rk    n float32 or NULL: r_k, the distance to the Ndens-th entry.
 * Distances are minimum-image, fp32 (fp64 when pos_is_f64) with one
 * rounding per component difference.  Requires n >= n_dens.
 */
int hop_density(hop_ctx *ctx, const void *pos, int64_t n, const hop_params *params,
                uint32_t *nbr, int32_t ld_nbr, float *dens, float *rk);

/*
 * Steps 2-3 (Sec. 2): hop to the densest of the first n_hop entries of each
 * row of nbr (density desc, then smaller index; the particle itself may win),
 * then follow hops to the root (a particle that is its own hop).
 *   dens n float32, nbr n x ld_nbr uint32 (as written by hop_density),
 *   hop n uint32 (may be NULL), chain n uint32 = index of the root.
 * Fails with HOP_ETIMEOUT if following does not end (lists without self).
 */
int hop_link(hop_ctx *ctx, const float *dens, const uint32_t *nbr, int32_t ld_nbr,
             int64_t n, int32_t n_hop, uint32_t *hop, uint32_t *chain);

/*
 * Merging step 3 (Sec. 2): boundary densities between chains.  For every i
 * with dens_i >= delta_outer and every j among the first n_merge entries of
 * row i, j != i, dens_j >= delta_outer, chain_i != chain_j, the pair
 * {chain_i, chain_j} records s = (double)dens_i + (double)dens_j (twice the
 * pair's average density, exact in fp64); each pair keeps its maximum.
 *   edge_pair  cap uint64: (lo << 32) | hi with lo < hi the chain labels,
 *   edge_sum   cap float64: the pair's maximum s,
 * written in ascending edge_pair order.  *n_edges (host) = number of pairs.
 * If cap < *n_edges, nothing is written and HOP_ETABLE is returned.
 * Synchronises the stream (reads the pair count).
 */
int hop_boundaries(hop_ctx *ctx, const uint32_t *chain, const float *dens,
                   const uint32_t *nbr, int32_t ld_nbr, int64_t n, int32_t n_merge,
                   float delta_outer, uint64_t *edge_pair, double *edge_sum,
                   int64_t cap, int64_t *n_edges);

/*
 * The global boundary table of Parallel HOP (Sec. 3): every subvolume builds
 * its own table (hop_boundaries over the particles it owns), the tables are
 * gathered, and each chain pair keeps its largest boundary.  This call takes
 * the gathered list -- pairs may repeat, in any order -- and writes each
 * distinct pair once with its largest sum, in ascending pair order:
 *   pair_in  m_in uint64 (lo << 32) | hi, device;  sum_in  m_in float64 >= 0;
 *   edge_pair, edge_sum, cap, *n_edges  as in hop_boundaries (HOP_ETABLE
 *   when cap is too small).  Synchronises the stream.
 */
int hop_boundaries_reduce(hop_ctx *ctx, const uint64_t *pair_in, const double *sum_in, int64_t m_in,
                          uint64_t *edge_pair, double *edge_sum, int64_t cap, int64_t *n_edges);

/*
 * Density normalisation of a subvolume (Parallel HOP Sec. 3).  A subvolume
 * together with its padding is run as its own problem, but its densities
 * must be normalised to the mean density of the whole box: later
 * hop_density / hop_run calls on this context use n_norm in place of their
 * own n in delta_i = (L^3 / n) sum W (0 restores their own n).  The batched
 * call keeps each subvolume's own count.
 */
int hop_set_norm_count(hop_ctx *ctx, int64_t n_norm);

/*
 * Merging steps 1, 2, 4, 5 (Sec. 2, Fig. 1): chains whose peak density is
 * >= delta_peak are proto-halos; proto-halos whose boundary s >= 2
 * delta_saddle merge, transitively; every other chain joins the proto-halo
 * reached along its densest propagated boundary (the maximum spanning forest
 * of the boundary graph with all proto-halos contracted, edges ordered by
 * s desc, then lo, then hi); a chain that reaches none is in no group.
 *   group n int32: -1 if dens_i < delta_outer or i's chain is in no group;
 *   otherwise the group's rank when groups are ordered by their peak
 *   (density desc, index asc).  *n_groups (host) = number of groups.
 * Synchronises the stream.
 */
int hop_merge(hop_ctx *ctx, const uint32_t *chain, const float *dens, int64_t n,
              const uint64_t *edge_pair, const double *edge_sum, int64_t n_edges,
              float delta_outer, float delta_saddle, float delta_peak,
              int32_t *group, int64_t *n_groups);

/*
 * The whole method in one call: steps 1-4 run in the context's spatially
 * sorted order and only the results are written in the caller's order.
 *   pos    n x 3 (float32 or float64), device OR host memory (pinned or
 *          pageable; host buffers are copied in on the stream).
 *   dens   n float32, device or host, or NULL.
 *   group  n int32, device or host (as in hop_merge).
 *   nbr    n x ld_nbr uint32 device, or NULL (as in hop_density).
 *   chain  n uint32 device, or NULL (as in hop_link).
 *   n_groups (host) number of groups.
 * Synchronises the stream.  Output is identical for every radius_mode.
 */
int hop_run(hop_ctx *ctx, const void *pos, int64_t n, const hop_params *params,
            float *dens, int32_t *group, int64_t *n_groups,
            uint32_t *nbr, int32_t ld_nbr, uint32_t *chain);

/*
 * Many independent periodic subvolumes in one pass (Parallel HOP Sec. 3
 * runs subvolumes as separate tasks; here they are independent problems
 * run together).  Subvolume b holds particles [offsets[b], offsets[b+1])
 * of pos, in its own periodic box [0, boxes[b])^3.  Each subvolume's
 * result is exactly that of hop_run on it alone: the same densities, the
 * same neighbour lists (offset by offsets[b]), the same group ids.
 *   pos      N x 3 float32 (N = offsets[B]), device or host memory.
 *   offsets  B + 1 int64 (host), offsets[0] = 0, every subvolume holding at
 *            least n_dens particles; N < 2^31 - 1.
 *   boxes    B float64 (host), each > 0.  params->box is not used and
 *            params->pos_is_f64 must be 0.
 *   dens     N float32, device or host, or NULL.
 *   group    N int32, device or host: -1, or the rank of the particle's
 *            group within its own subvolume (ordered as in hop_merge).
 *   n_groups B int64 (host): groups per subvolume.
 *   nbr      N x ld_nbr uint32 device (indices into the whole batch), or NULL.
 *   flags    0: the pass is captured into a CUDA graph (kept by the context
 *            and replayed while the subvolumes, parameters, tuning and
 *            buffers stay the same); HOP_BATCH_EAGER: kernels are enqueued
 *            one by one and the merge loops are driven from the host.
 * Queries per warp must be 4, 8, 16 or 32 (hop_set_tuning; 32 runs one
 * query per lane); with HOP_RADIUS_LEARNED the network loaded for that
 * setting is used.  Stage
 * times in hop_stats are those of the pass on the device.  Synchronises the
 * stream.
 */
#define HOP_BATCH_EAGER 1
int hop_run_batch(hop_ctx *ctx, const float *pos, const int64_t *offsets, const double *boxes,
                  int32_t B, const hop_params *params, float *dens, int32_t *group,
                  int64_t *n_groups, uint32_t *nbr, int32_t ld_nbr, int32_t flags);

/* Tuning of the kNN search: queries per warp (the lanes of a warp split
 * into 32 / qpw lanes per query), search cells per radius (the cell side is
 * about radius / cpr), and the per-query candidate buffer in units of
 * n_dens (buf_factor 2, 3 or 4; 0 = 4 up to 4 queries per warp, else 3).
 * ms is the autotuner's measured pass time (-1 if the candidate was
 * skipped). */
typedef struct hop_tuning {
    int32_t qpw, cpr, buf_factor;
    float ms;
} hop_tuning;
int hop_get_tuning(const hop_ctx *ctx, hop_tuning *out);
int hop_apply_tuning(hop_ctx *ctx, const hop_tuning *t);

/*
 * Times the batched pass (graph replays, median of reps) for each of n_cand
 * candidates on the given batch, writes each candidate's ms, and applies
 * the fastest; *best = its index.  Candidates with a qpw other than 4, 8,
 * 16 or 32, or (learned radius) with no network loaded for their qpw, are
 * skipped.  Results do not depend on the tuning.  Synchronises the stream.
 */
int hop_autotune(hop_ctx *ctx, const float *pos, const int64_t *offsets, const double *boxes,
                 int32_t B, const hop_params *params, hop_tuning *cand, int32_t n_cand,
                 int32_t reps, int32_t *best);

/*
 * hop_link without any device allocation.  (No counterpart in the paper:
 * this is an interface for callers, not part of the method.)
 *
 * Some callers cannot call cudaMalloc.  For example, a host program may give
 * all device memory to its own pool allocator and forbid other
 * allocations.  A latency-bound loop may not afford one either, because a
 * device allocation can synchronise the device.  Such callers cannot create
 * a hop_ctx, whose scratch memory grows on demand.  This call computes
 * exactly what hop_link computes (same hops, same chain labels, same
 * errors).  It keeps its scratch, the per-particle density keys and an error
 * word, in one array in this library's own device memory:
 * HOP_STATIC_LINK_MAX_N * 8 + 256 bytes (8 MiB + 256 B).  Every GPU that
 * loads the library holds that array until the process exits.
 *   dens, nbr, ld_nbr, n, n_hop  as in hop_link (device pointers);
 *   hop, chain  n uint32 each, device, both required;
 *   cuda_stream  the stream to enqueue on (NULL = legacy default stream).
 * Returns HOP_ESTATIC without touching any buffer when n > the maximum.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  Make that first call before any stream
 * capture.  The array is shared by every call on a device and keeps the last
 * call's contents.  Calls that overlap on the GPU (different streams or
 * threads, not ordered by the caller) race on it and give wrong results.
 * Like hop_link, the call synchronises the stream to read its error word.
 */
#define HOP_STATIC_LINK_MAX_N (1 << 20)
int hop_link_static(const float *dens, const uint32_t *nbr, int32_t ld_nbr, int64_t n,
                    int32_t n_hop, uint32_t *hop, uint32_t *chain, void *cuda_stream);

/*
 * Halo statistics.  Once the halos are known, Parallel HOP computes for each
 * its dark matter mass, centre of mass and maximum radius (Sec. 3, end of
 * the merging description).  Particle masses are equal, so a halo's mass
 * is its member count.  In the periodic box the centre of mass is taken
 * about the halo's peak particle (its densest member, then the smaller
 * index): the members' minimum-image offsets from the peak are averaged and
 * added to the peak's position, then wrapped into [0, box).  The maximum
 * radius is the largest minimum-image distance from that centre to a
 * member.  Coordinates are taken in fixed point (2^-32 of the box, rounded
 * once), so centres are reproducible and within 2^-33 of the box of the
 * exact mean, and radii within 1.5 x 2^-32 of the box of the exact
 * distance.  All pointers are device memory, in the caller's order:
 *   pos    n x 3 float32 (float64 if pos_is_f64), as given to hop_run;
 *   dens   n float32; group n int32 (-1 = no halo, else < n_groups);
 *   count  n_groups int64, peak n_groups uint32 (particle index),
 *   com    n_groups x 3 float64, rmax n_groups float64 (outputs).
 * A group id >= n_groups is HOP_EINVAL.  Synchronises the stream;
 * hop_get_stats reports the time in ms_total.
 */
int hop_halo_stats(hop_ctx *ctx, const void *pos, int32_t pos_is_f64, const float *dens,
                   const int32_t *group, int64_t n, int64_t n_groups, double box,
                   int64_t *count, uint32_t *peak, double *com, double *rmax);

/*
 * ADAPTAHOP subhalos (Parallel HOP Sec. 6, "Parallel HOP and Subhalos"),
 * from HOP's own densities, neighbour lists and chains:
 *   1. symmetric boundaries: chains a and b share a boundary only when a
 *      particle of a has a particle of b among the first n_merge entries of
 *      its row AND a particle of b has one of a there (both particles >=
 *      delta_outer, as in hop_boundaries).  Its value s is the largest
 *      (double)dens_i + (double)dens_j over the links of both directions;
 *   2. for every threshold delta_s = levels[l]: boundaries with
 *      s < 2 delta_s are destroyed, and chains joined by the rest merge,
 *      transitively.  A particle with dens_i >= delta_s belongs to its
 *      merged set's subhalo;
 *   3. a subhalo of N members is rejected when N < n_min, or when its
 *      members' mean density (fp64 sum / N) is below
 *      delta_s * (1 + f_poisson / sqrt(N)): the Poisson noise of a count
 *      of N, scaled by f_poisson (0 keeps every subhalo);
 *   4. the accepted subhalos of a level are ranked by their peak member
 *      (density desc, index asc).
 *   chain, dens, nbr, ld_nbr, n, n_merge, delta_outer  as in hop_boundaries
 *            (device memory, caller's order; chain labels are roots);
 *   levels   n_levels float32, HOST memory, each finite and >= delta_outer,
 *            in any order;
 *   sub      n_levels x n int32, device: sub[l * n + i] = the rank of i's
 *            subhalo at levels[l], or -1;
 *   n_sub    n_levels int64, host: subhalos per level.
 * Under one threshold below another, every subhalo of the higher one lies
 * within a single merged set of the lower (a hierarchy).  Runs the levels
 * one after another.  Synchronises the stream.  hop_get_stats reports
 * ms_total, ms_boundaries (step 1), ms_merge (the rest: chain ids and the
 * levels), n_chains (chains above delta_outer) and n_edges (symmetric
 * boundaries).
 */
int hop_subhalos(hop_ctx *ctx, const uint32_t *chain, const float *dens, const uint32_t *nbr,
                 int32_t ld_nbr, int64_t n, int32_t n_merge, float delta_outer, const float *levels,
                 int32_t n_levels, int64_t n_min, double f_poisson, int32_t *sub, int64_t *n_sub);

/* Counters and stage times (ms, CUDA events on the context stream) of the
 * last hop_run / hop_density call. */
typedef struct hop_stats {
    double ms_sort, ms_radius, ms_knn, ms_link, ms_boundaries, ms_merge, ms_total;
    int64_t candidates;      /* (query, candidate) distance evaluations          */
    int64_t searches;        /* warp searches started (first tries + retries)    */
    int64_t retries;         /* searches repeated with a larger radius           */
    int64_t warps;           /* warp tasks (query chunks)                         */
    int64_t n_chains, n_edges, n_groups;
    int32_t knn_queries_per_warp, knn_cells_per_radius;
    int64_t launches;        /* kernels this library launched during the call     */
} hop_stats;
int hop_get_stats(const hop_ctx *ctx, hop_stats *out);

/*
 * Learned search radius (a 3-layer MLP, 27 -> 64 -> 64 -> 1, ReLU).
 * Input: log(1 + count) of the 27 cells of the 3x3x3 stencil around a
 * query chunk's cell, at the level whose cell size just covers the chunk.
 * Output: log(R / cell size), R the largest Ndens-th-neighbour distance of
 * the chunk.  Weights are BF16, accumulation FP32 (fp32 master copy for
 * training).  The parameter vector layout is
 *   W1[64][27], b1[64], W2[64][64], b2[64], W3[64], b3[1]   (HOP_MLP_NPARAM).
 */
#define HOP_MLP_IN 27
#define HOP_MLP_HID 64
#define HOP_MLP_NPARAM (64 * 27 + 64 + 64 * 64 + 64 + 64 + 1)

/* Loads fp32 parameters (host) and the radius margin added to the predicted
 * log radius before the search.  A context keeps one network per
 * queries-per-warp setting (the chunk features depend on it): this call,
 * and the other hop_mlp_* calls, act on the network of the current
 * setting (hop_set_tuning). */
int hop_mlp_load(hop_ctx *ctx, const float *params_host, float log_margin);
/* Copies the current fp32 master parameters to the host. */
int hop_mlp_get(hop_ctx *ctx, float *params_host);

/* After a hop_run or hop_density on pos, writes one training sample per
 * query chunk: feat (n_chunks x 27 float32, device) and target (n_chunks
 * float32, device) = log(max r_k over the chunk / cell size).  *n_chunks
 * (host) is the number of samples; cap is the capacity of both buffers.
 * Synchronises the stream. */
int hop_mlp_samples(hop_ctx *ctx, float *feat, float *target, int64_t cap, int64_t *n_chunks);

/* Forward pass over m samples (device): out[m] float32. */
int hop_mlp_forward(hop_ctx *ctx, const float *feat, int64_t m, float *out);

/* Mean-squared-error gradient over m samples (device): loss (host) and grad
 * (HOP_MLP_NPARAM float32, device), both averaged over the samples, at the
 * current BF16 weights. */
int hop_mlp_grad(hop_ctx *ctx, const float *feat, const float *target, int64_t m,
                 double *loss, float *grad);

/* Trains in place with Adam (lr, beta1 0.9, beta2 0.999) on mini-batches of
 * `batch` samples for `epochs` passes over the (device) data, from a
 * deterministic sample order given by `seed`.  *final_loss (host) is the mean
 * loss of the last epoch.  Synchronises the stream. */
int hop_mlp_train(hop_ctx *ctx, const float *feat, const float *target, int64_t m,
                  int32_t epochs, int32_t batch, float lr, uint64_t seed, double *final_loss);

#ifdef __cplusplus
}
#endif

#endif /* HOP_H_ */
