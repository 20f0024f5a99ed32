// Batched HOP: many independent periodic subvolumes (each its own box and
// particle count) in one pass, captured once into a CUDA graph and replayed.
//
// Parallel HOP splits one volume into subvolumes so that separate CPU tasks
// can run HOP side by side (Sec. 3); here the subvolumes are independent
// problems and the GPU runs all of them at once.  Every stage of the single
// pass runs over the concatenation of the subvolumes:
//   - the sort key leads with the subvolume number, so one radix sort puts
//     each subvolume's particles in a contiguous range, Morton-ordered in
//     its own box; every subvolume gets its own dense cell table;
//   - one persistent kNN launch takes query chunks from all subvolumes off
//     a shared counter (chunks never straddle two subvolumes), each chunk
//     using its subvolume's box, table, first radius and normalisation;
//   - hops, chains, boundaries and the merge need no change: neighbours
//     never cross subvolumes, so the chain forest and the boundary graph
//     split into per-subvolume parts by themselves; group ranks are taken
//     within each subvolume;
//   - every data-dependent size (chains, edges, groups) stays on the device
//     and the merge rounds are conditional while nodes, so the pass has no
//     host round trip and is captured as one graph.
// A subvolume's densities, neighbour lists and group ids are those of
// hop_run on that subvolume alone (indices offset by its first particle).
#include "hop_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

// End of one round of a device-bounded loop: count the round; with a graph
// handle, set the loop condition (and clear the round flag for the next
// round); without one, leave the flag for the host to read.
__global__ void loop_cond_kernel(cudaGraphConditionalHandle h, int use_handle, uint32_t *changed,
                                 uint32_t *round, int max_rounds, uint32_t *err, uint32_t err_bit)
{
    const uint32_t r = ++*round;
    bool go = *changed != 0u;
    if (go && r >= (uint32_t)max_rounds) {
        atomicOr(err, err_bit);
        go = false;
    }
    if (use_handle) {
        *changed = 0u;
        cudaGraphSetConditional(h, go ? 1u : 0u);
    } else if (!go) {
        *changed = 0u;
    }
}

// Restores the context's stream when a capture of a loop body ends early.
struct StreamSwap {
    hop_ctx *c;
    cudaStream_t saved;
    StreamSwap(hop_ctx *ctx, cudaStream_t s) : c(ctx), saved(ctx->stream) { c->stream = s; }
    ~StreamSwap() { c->stream = saved; }
};

}  // namespace

int graph_while(hop_ctx *c, uint32_t *changed, uint32_t *round, int max_rounds, uint32_t err_bit,
                int (*body)(hop_ctx *, void *), void *arg)
{
    if (!c->capturing) {
        uint32_t *h = (uint32_t *)c->h_pinned + 256;
        for (int it = 0; it <= max_rounds; ++it) {
            int rc = body(c, arg);
            if (rc) return rc;
            loop_cond_kernel<<<1, 1, 0, c->stream>>>(0, 0, changed, round, max_rounds, c->d_err, err_bit);
            HOP_LAUNCH(c);
            HOP_CUDA(c, cudaMemcpyAsync(h, changed, 4, cudaMemcpyDeviceToHost, c->stream));
            HOP_CUDA(c, cudaStreamSynchronize(c->stream));
            if (!h[0]) break;
            HOP_CUDA(c, cudaMemsetAsync(changed, 0, 4, c->stream));
        }
        return HOP_OK;
    }
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    HOP_CUDA(c, cudaStreamGetCaptureInfo(c->stream, &st, nullptr, &g, &deps, nullptr, &nd));
    if (st != cudaStreamCaptureStatusActive) return ctx_fail(c, HOP_ECUDA, "no capture open for a graph loop");
    cudaGraphConditionalHandle handle;
    HOP_CUDA(c, cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    HOP_CUDA(c, cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    cudaGraph_t body_graph = np.conditional.phGraph_out[0];
    HOP_CUDA(c, cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1,
                                                     cudaStreamSetCaptureDependencies));
    if (!c->side) HOP_CUDA(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    HOP_CUDA(c, cudaStreamBeginCaptureToGraph(c->side, body_graph, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed));
    int rc;
    {
        StreamSwap swap(c, c->side);
        rc = body(c, arg);
        if (rc == HOP_OK) {
            loop_cond_kernel<<<1, 1, 0, c->stream>>>(handle, 1, changed, round, max_rounds, c->d_err, err_bit);
            ++c->launches;
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = ctx_cuda(c, e, "kernel launch");
        }
    }
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->side, &out);
    if (rc) return rc;
    HOP_CUDA(c, e);
    return HOP_OK;
}

// ------------------------------------------------------------ the pass ---
struct BatchGraph {
    // everything the captured graph depends on
    std::vector<int64_t> offsets;
    std::vector<double> boxes;
    hop_params params{};
    int qpw = 0, cpr = 0, capf = 0;
    const void *mlp_w = nullptr;
    float mlp_margin = 0.f;
    const float *dpos = nullptr;
    float *dens = nullptr;
    int32_t *group = nullptr;
    uint32_t *nbr = nullptr;
    int ld_nbr = 0;
    int64_t table_cap = 0;
    int64_t chain_cap = 0;
    uint64_t epoch = 0;
    // the graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> graveyard;   // buffers replaced while capturing
    int64_t captured_kernels = 0;    // loop bodies counted once
};

namespace {

constexpr int kProtoBodyKernels = 3;     // hook, compress, loop condition
constexpr int kBoruvkaBodyKernels = 6;   // fill, best edge, target, hook, compress, loop condition

// Host-side description of one batched pass.
struct BatchPlan {
    int B = 0;
    int64_t n = 0, n_chunks = 0, n_cells = 0;
    std::vector<SegDesc> seg;
};

int make_plan(hop_ctx *c, const int64_t *offsets, const double *boxes, int B, const hop_params *p,
              int qpw, BatchPlan *pl)
{
    if (B < 1 || B > 65536) return ctx_fail(c, HOP_EINVAL, "number of subvolumes must be in [1, 65536]");
    if (!offsets || !boxes) return ctx_fail(c, HOP_EINVAL, "offsets and boxes are required");
    if (offsets[0] != 0) return ctx_fail(c, HOP_EINVAL, "offsets[0] must be 0");
    pl->B = B;
    pl->seg.resize(B);
    int64_t chunks = 0, cells = 0;
    for (int b = 0; b < B; ++b) {
        const int64_t nb = offsets[b + 1] - offsets[b];
        if (nb < p->n_dens) return ctx_fail(c, HOP_EINVAL, "every subvolume needs at least n_dens particles");
        const double box = boxes[b];
        if (!(box > 0) || !std::isfinite(box)) return ctx_fail(c, HOP_EINVAL, "every box must be positive");
        SegDesc &d = pl->seg[b];
        d.base = offsets[b];
        d.n = nb;
        d.chunk0 = chunks;
        d.cell0 = cells;
        d.box = box;
        d.norm = box * box * box / ((double)nb * 3.14159265358979323846);
        d.plain_r = plain_radius_for(nb, box, p->n_dens);
        d.level_dense = dense_level_for(nb);
        chunks += (nb + qpw - 1) / qpw;
        cells += (int64_t(1) << (3 * d.level_dense)) + 1;
    }
    pl->n = offsets[B];
    if (pl->n >= (int64_t(1) << 31) - 1) return ctx_fail(c, HOP_EINVAL, "total particles must be < 2^31 - 1");
    pl->n_chunks = chunks;
    pl->n_cells = cells;
    return HOP_OK;
}

// Device words of a pass: merge counts (8), edge count, spare, boundary
// insert counter (u64), then the per-subvolume group counts.
struct PassWords {
    uint32_t *counts, *m_dev, *n_groups;
    unsigned long long *nins;
};

int pass_words(hop_ctx *c, int B, PassWords *w)
{
    char *p = (char *)ctx_buf(c, S_BATCH, 64 + (size_t)B * 4);
    if (!p) return HOP_ENOMEM;
    w->counts = (uint32_t *)p;
    w->m_dev = (uint32_t *)(p + 32);
    w->nins = (unsigned long long *)(p + 40);
    w->n_groups = (uint32_t *)(p + 64);
    return HOP_OK;
}

int record(hop_ctx *c, int i)
{
    if (c->capturing)
        HOP_CUDA(c, cudaEventRecordWithFlags(c->ev[i], c->stream, cudaEventRecordExternal));
    else
        HOP_CUDA(c, cudaEventRecord(c->ev[i], c->stream));
    return HOP_OK;
}

// Enqueues the whole pass on the context's stream (captured or not).
int enqueue_pass(hop_ctx *c, const BatchPlan &pl, const SegDesc *seg, const PassWords &w,
                 const hop_params *p, const float *dpos, float *dens, int32_t *group, uint32_t *nbr,
                 int ld_nbr, int64_t table_cap, int64_t chain_cap)
{
    const int64_t n = pl.n;
    int rc;
    HOP_CUDA(c, cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * 16, c->stream));
    if ((rc = record(c, 0))) return rc;
    void *spos;
    uint32_t *perm, *cellT;
    uint64_t *keys;
    rc = grid_build_seg(c, dpos, n, seg, pl.B, pl.n_cells, &spos, &perm, &keys, &cellT);
    if (rc) return rc;
    if ((rc = record(c, 1))) return rc;
    float *chunk_r = nullptr;
    if (p->radius_mode != HOP_RADIUS_PLAIN) {
        chunk_r = (float *)ctx_buf(c, S_CHUNK_R, pl.n_chunks * sizeof(float));
        if (!chunk_r) return HOP_ENOMEM;
        if (p->radius_mode == HOP_RADIUS_COUNT)
            rc = chunk_radius_seg(c, spos, keys, cellT, seg, pl.B, pl.n_chunks, c->qpw, p->n_dens, chunk_r);
        else
            rc = mlp_radius_seg(c, spos, keys, cellT, seg, pl.B, pl.n_chunks, c->qpw, p->n_dens, chunk_r);
        if (rc) return rc;
    }
    if ((rc = record(c, 2))) return rc;
    const int n_out = std::max<int>(p->n_hop, nbr ? ld_nbr : 0);
    uint32_t *nbr_s = (uint32_t *)ctx_buf(c, S_NBR_S, (size_t)n * n_out * sizeof(uint32_t));
    float *dens_s = (float *)ctx_buf(c, S_DENS_S, n * sizeof(float));
    if (!nbr_s || !dens_s) return HOP_ENOMEM;
    KnnArgs a;
    a.spos = spos;
    a.keys = keys;
    a.cellT = cellT;
    a.level_dense = 0;
    a.n = n;
    a.box = 1.0;
    a.k = p->n_dens;
    a.n_out = n_out;
    a.ld_out = n_out;
    a.chunk_r = chunk_r;
    a.plain_r = 0.f;
    a.nbr_s = nbr_s;
    a.dens_s = dens_s;
    a.rk_s = nullptr;
    a.seg = seg;
    a.B = pl.B;
    a.n_chunks = pl.n_chunks;
    if (pl.B == 1) {
        // one subvolume: the kernel without per-chunk descriptors, with the
        // same box, table, radius and normalisation as kernel arguments
        a.seg = nullptr;
        a.level_dense = pl.seg[0].level_dense;
        a.box = pl.seg[0].box;
        a.plain_r = pl.seg[0].plain_r;
    }
    rc = knn_launch(c, a, false, c->qpw, c->cpr);
    if (rc) return rc;
    if ((rc = record(c, 3))) return rc;
    uint64_t *dkey = (uint64_t *)ctx_buf(c, S_DKEY, n * sizeof(uint64_t));
    uint32_t *hop_s = (uint32_t *)ctx_buf(c, S_HOP, n * sizeof(uint32_t));
    uint32_t *chain_s = (uint32_t *)ctx_buf(c, S_CHAIN, n * sizeof(uint32_t));
    int32_t *group_s = (int32_t *)ctx_buf(c, S_GROUP_OUT, n * sizeof(int32_t));
    if (!dkey || !hop_s || !chain_s || !group_s) return HOP_ENOMEM;
    if ((rc = make_dkey(c, dens_s, perm, n, dkey))) return rc;
    if ((rc = hop_links_async(c, dkey, nbr_s, n_out, n, p->n_hop, hop_s, chain_s))) return rc;
    if ((rc = record(c, 5))) return rc;
    uint64_t *ek;
    double *es;
    rc = boundaries_table_async(c, chain_s, dkey, nbr_s, n_out, n, p->n_merge, p->delta_outer, table_cap,
                                w.m_dev, w.nins, &ek, &es);
    if (rc) return rc;
    if ((rc = record(c, 6))) return rc;
    MergeGraphArgs ma;
    ma.chain = chain_s;
    ma.dkey = dkey;
    ma.n = n;
    ma.edge_key = ek;
    ma.edge_sum = es;
    ma.m = DevCount{table_cap, w.m_dev};
    ma.d_o = p->delta_outer;
    ma.d_s = p->delta_saddle;
    ma.d_p = p->delta_peak;
    ma.seg = seg;
    ma.B = pl.B;
    ma.group = group_s;
    ma.n_groups = w.n_groups;
    ma.counts = w.counts;
    ma.c_cap = chain_cap;
    if ((rc = merge_groups_graph(c, ma))) return rc;
    if ((rc = record(c, 7))) return rc;
    rc = scatter_outputs(c, perm, n, dens_s, dens, group_s, group, nbr_s, n_out, nbr, ld_nbr,
                         nbr ? ld_nbr : 0, nullptr, nullptr);
    if (rc) return rc;
    return record(c, 9);
}

void graph_drop(hop_ctx *c)
{
    BatchGraph *g = c->batch;
    if (!g) return;
    cudaStreamSynchronize(c->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (void *p : g->graveyard) cudaFree(p);
    delete g;
    c->batch = nullptr;
}

bool graph_matches(const hop_ctx *c, const BatchGraph *g, const int64_t *offsets, const double *boxes,
                   int B, const hop_params *p, const float *dpos, float *dens, int32_t *group,
                   uint32_t *nbr, int ld_nbr)
{
    if (!g || !g->exec) return false;
    if ((int)g->boxes.size() != B || g->epoch != c->buf_epoch) return false;
    if (std::memcmp(&g->params, p, sizeof(hop_params)) != 0) return false;
    if (g->qpw != c->qpw || g->cpr != c->cpr || g->capf != c->capf) return false;
    if (p->radius_mode == HOP_RADIUS_LEARNED &&
        (g->mlp_w != c->mlp->w16 || g->mlp_margin != c->mlp->log_margin))
        return false;
    if (g->dpos != dpos || g->dens != dens || g->group != group || g->nbr != nbr || g->ld_nbr != ld_nbr)
        return false;
    return std::equal(g->offsets.begin(), g->offsets.end(), offsets) &&
           std::equal(g->boxes.begin(), g->boxes.end(), boxes);
}

}  // namespace

void batch_free(hop_ctx *c) { graph_drop(c); }

namespace {

bool host_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

int check_batch_params(hop_ctx *c, const hop_params *p)
{
    if (!p) return ctx_fail(c, HOP_EINVAL, "params is NULL");
    if (p->n_dens < 2 || p->n_dens > kMaxDens) return ctx_fail(c, HOP_EINVAL, "n_dens must be in [2, 128]");
    if (p->n_hop < 1 || p->n_hop > p->n_dens) return ctx_fail(c, HOP_EINVAL, "n_hop must be in [1, n_dens]");
    if (p->n_merge < 1 || p->n_merge > p->n_hop) return ctx_fail(c, HOP_EINVAL, "n_merge must be in [1, n_hop]");
    if (p->pos_is_f64) return ctx_fail(c, HOP_EINVAL, "batched passes take float32 positions");
    if (p->radius_mode < HOP_RADIUS_PLAIN || p->radius_mode > HOP_RADIUS_LEARNED)
        return ctx_fail(c, HOP_EINVAL, "unknown radius_mode");
    if (p->radius_mode == HOP_RADIUS_LEARNED && !c->mlp->loaded)
        return ctx_fail(c, HOP_ENOMODEL, "no radius network loaded for this queries-per-warp setting");
    if (c->qpw != 4 && c->qpw != 8 && c->qpw != 16 && c->qpw != 32)
        return ctx_fail(c, HOP_EINVAL, "batched passes take 4, 8, 16 or 32 queries per warp");
    return HOP_OK;
}

// Captures the pass into a new graph (replacing the cached one).
int capture_pass(hop_ctx *c, const BatchPlan &pl, const SegDesc *seg, const PassWords &w,
                 const hop_params *p, const float *dpos, float *dens, int32_t *group, uint32_t *nbr,
                 int ld_nbr, int64_t table_cap, int64_t chain_cap, const int64_t *offsets,
                 const double *boxes)
{
    graph_drop(c);
    BatchGraph *g = new BatchGraph();
    c->batch = g;
    g->offsets.assign(offsets, offsets + pl.B + 1);
    g->boxes.assign(boxes, boxes + pl.B);
    g->params = *p;
    g->qpw = c->qpw;
    g->cpr = c->cpr;
    g->capf = c->capf;
    g->mlp_w = c->mlp->w16;
    g->mlp_margin = c->mlp->log_margin;
    g->dpos = dpos;
    g->dens = dens;
    g->group = group;
    g->nbr = nbr;
    g->ld_nbr = ld_nbr;
    g->table_cap = table_cap;
    g->chain_cap = chain_cap;
    const int64_t l0 = c->launches;
    if (!c->side) HOP_CUDA(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    if (!c->cap) HOP_CUDA(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    // capture on the context's own stream (the legacy default stream cannot
    // be captured); the graph is launched on the caller's stream
    int rc;
    cudaError_t e;
    cudaGraph_t graph = nullptr;
    {
        StreamSwap swap(c, c->cap);
        HOP_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        c->capturing = true;
        c->graveyard.clear();
        rc = enqueue_pass(c, pl, seg, w, p, dpos, dens, group, nbr, ld_nbr, table_cap, chain_cap);
        c->capturing = false;
        g->graveyard.swap(c->graveyard);
        e = cudaStreamEndCapture(c->stream, &graph);
    }
    g->graph = graph;
    if (rc) return rc;
    HOP_CUDA(c, e);
    HOP_CUDA(c, cudaGraphInstantiate(&g->exec, graph, 0));
    g->captured_kernels = c->launches - l0;
    g->epoch = c->buf_epoch;
    return HOP_OK;
}

void read_knn_counters(hop_ctx *c)
{
    unsigned long long h[kCntNum] = {0};
    cudaMemcpy(h, c->d_counters, sizeof(h), cudaMemcpyDeviceToHost);
    c->stats.candidates = (int64_t)h[kCntCand];
    c->stats.searches = (int64_t)h[kCntSearch];
    c->stats.retries = (int64_t)h[kCntRetry];
    c->stats.warps = (int64_t)h[kCntWarps];
    c->stats.knn_queries_per_warp = c->qpw;
    c->stats.knn_cells_per_radius = c->cpr;
}

double ev_span(hop_ctx *c, int a, int b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return ms;
}

}  // namespace

extern "C" {

int hop_run_batch(hop_ctx *c, const float *pos, const int64_t *offsets, const double *boxes, int32_t B,
                  const hop_params *p, float *dens, int32_t *group, int64_t *n_groups, uint32_t *nbr,
                  int32_t ld_nbr, int32_t flags)
{
    if (!c) return HOP_EINVAL;
    c->err.clear();
    int rc = check_batch_params(c, p);
    if (rc) return rc;
    if (!pos || !group || !n_groups) return ctx_fail(c, HOP_EINVAL, "pos, group and n_groups are required");
    if (nbr && (ld_nbr < p->n_hop || ld_nbr > p->n_dens))
        return ctx_fail(c, HOP_EINVAL, "ld_nbr must be in [n_hop, n_dens]");
    if (flags & ~HOP_BATCH_EAGER) return ctx_fail(c, HOP_EINVAL, "unknown flags");
    BatchPlan pl;
    if ((rc = make_plan(c, offsets, boxes, B, p, c->qpw, &pl))) return rc;
    HOP_CUDA(c, cudaSetDevice(c->device));
    const int64_t n = pl.n;
    if (nbr && host_ptr(nbr)) return ctx_fail(c, HOP_EINVAL, "nbr must be device memory");
    const bool host_pos = host_ptr(pos), host_dens = dens && host_ptr(dens), host_group = host_ptr(group);
    const float *dpos = pos;
    float *dens_dev = dens;
    int32_t *group_dev = group;
    if (host_pos) {
        dpos = (const float *)ctx_buf(c, S_POS_IN, n * 3 * sizeof(float));
        if (!dpos) return HOP_ENOMEM;
    }
    if (host_dens && !(dens_dev = (float *)ctx_buf(c, S_OUT_DENS, n * sizeof(float)))) return HOP_ENOMEM;
    if (host_group && !(group_dev = (int32_t *)ctx_buf(c, S_OUT_GROUP, n * sizeof(int32_t)))) return HOP_ENOMEM;
    SegDesc *seg = (SegDesc *)ctx_buf(c, S_SEG, (size_t)B * sizeof(SegDesc));
    PassWords w;
    if (!seg || (rc = pass_words(c, B, &w))) return seg ? rc : HOP_ENOMEM;
    const bool eager = (flags & HOP_BATCH_EAGER) != 0;
    const int64_t launches0 = c->launches;
    HOP_CUDA(c, cudaEventRecord(c->ev[8], c->stream));
    if (host_pos)
        HOP_CUDA(c, cudaMemcpyAsync((void *)dpos, pos, n * 3 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    // capacities of the boundary table and of the merge's chain arrays:
    // first guesses well above the chain pairs and chains above delta_outer
    // that halo boxes have (n / 16), grown when the pass reports an overflow
    int64_t cap = int64_t(1) << 12;
    while (cap < n / 16 && cap < (int64_t(1) << 31)) cap <<= 1;
    int64_t ccap = std::min<int64_t>(n, n / 16 + 65536);
    if (!eager && c->batch && c->batch->table_cap > cap) cap = c->batch->table_cap;
    if (!eager && c->batch && c->batch->chain_cap > ccap) ccap = c->batch->chain_cap;
    std::vector<uint32_t> hw(16 + B);
    uint32_t herr = 0;
    for (int attempt = 0; attempt < 6; ++attempt) {
        const bool fresh = eager || !graph_matches(c, c->batch, offsets, boxes, B, p, dpos, dens_dev, group_dev,
                                                   nbr, ld_nbr) || c->batch->table_cap != cap ||
                           c->batch->chain_cap != ccap;
        if (fresh) {
            // descriptors for this plan (the graph reads them at run time)
            HOP_CUDA(c, cudaMemcpyAsync(seg, pl.seg.data(), (size_t)B * sizeof(SegDesc), cudaMemcpyHostToDevice,
                                        c->stream));
            HOP_CUDA(c, cudaStreamSynchronize(c->stream));
        }
        if (eager) {
            rc = enqueue_pass(c, pl, seg, w, p, dpos, dens_dev, group_dev, nbr, ld_nbr, cap, ccap);
            if (rc) return rc;
        } else {
            if (fresh) {
                rc = capture_pass(c, pl, seg, w, p, dpos, dens_dev, group_dev, nbr, ld_nbr, cap, ccap, offsets,
                                  boxes);
                if (rc) {
                    graph_drop(c);
                    return rc;
                }
            }
            HOP_CUDA(c, cudaGraphLaunch(c->batch->exec, c->stream));
        }
        HOP_CUDA(c, cudaMemcpyAsync(hw.data(), w.counts, 8 * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
        HOP_CUDA(c, cudaMemcpyAsync(hw.data() + 8, w.m_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
        HOP_CUDA(c, cudaMemcpyAsync(hw.data() + 16, w.n_groups, (size_t)B * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, c->stream));
        HOP_CUDA(c, cudaMemcpyAsync(&herr, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
        HOP_CUDA(c, cudaStreamSynchronize(c->stream));
        if ((herr & ~(kErrTableFull | kErrChainCap)) == 0 && herr != 0 && attempt < 5) {
            // the boundary table or the chain arrays overflowed: larger ones,
            // a new capture (the last attempt keeps the error word for the
            // report below)
            HOP_CUDA(c, cudaMemsetAsync(c->d_err, 0, 4, c->stream));
            if (herr & kErrTableFull) cap <<= 2;
            if (herr & kErrChainCap) ccap = std::min<int64_t>(n, ccap * 4);
            continue;
        }
        break;
    }
    rc = ctx_check_device_error(c);
    if (rc) return rc;
    if (host_dens)
        HOP_CUDA(c, cudaMemcpyAsync(dens, dens_dev, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (host_group)
        HOP_CUDA(c, cudaMemcpyAsync(group, group_dev, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    HOP_CUDA(c, cudaEventRecord(c->ev[10], c->stream));
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    int64_t total_groups = 0;
    for (int b = 0; b < B; ++b) {
        n_groups[b] = hw[16 + b];
        total_groups += hw[16 + b];
    }
    read_knn_counters(c);
    c->stats.ms_sort = ev_span(c, 0, 1);
    c->stats.ms_radius = ev_span(c, 1, 2);
    c->stats.ms_knn = ev_span(c, 2, 3);
    c->stats.ms_link = ev_span(c, 3, 5);
    c->stats.ms_boundaries = ev_span(c, 5, 6);
    c->stats.ms_merge = ev_span(c, 6, 7);
    c->stats.ms_total = ev_span(c, 0, 9);   // the pass on the device, without host copies
    c->stats.n_chains = hw[0];
    c->stats.n_edges = hw[8];
    c->stats.n_groups = total_groups;
    if (eager) {
        c->stats.launches = c->launches - launches0;
    } else {
        // kernels the replay ran: the captured ones, plus the loop bodies'
        // repeats (hw[3], hw[4] rounds each)
        const int64_t r1 = hw[3], r2 = hw[4];
        c->stats.launches = c->batch->captured_kernels + std::max<int64_t>(r1 - 1, 0) * kProtoBodyKernels +
                            std::max<int64_t>(r2 - 1, 0) * kBoruvkaBodyKernels;
    }
    return HOP_OK;
}

int hop_get_tuning(const hop_ctx *c, hop_tuning *out)
{
    if (!c || !out) return HOP_EINVAL;
    out->qpw = c->qpw;
    out->cpr = c->cpr;
    out->buf_factor = c->capf;
    out->ms = 0.f;
    return HOP_OK;
}

int hop_apply_tuning(hop_ctx *c, const hop_tuning *t)
{
    if (!c || !t) return HOP_EINVAL;
    if (t->buf_factor != 0 && (t->buf_factor < 2 || t->buf_factor > 6))
        return ctx_fail(c, HOP_EINVAL, "buffer factor must be 0 (default) or 2 to 6");
    const int rc = hop_set_tuning(c, t->qpw, t->cpr);
    if (rc) return rc;
    c->capf = t->buf_factor;
    return HOP_OK;
}

int hop_autotune(hop_ctx *c, const float *pos, const int64_t *offsets, const double *boxes, int32_t B,
                 const hop_params *p, hop_tuning *cand, int32_t n_cand, int32_t reps, int32_t *best)
{
    if (!c || !cand || n_cand < 1 || !best) return HOP_EINVAL;
    c->err.clear();
    if (reps < 1) reps = 1;
    if (!offsets || B < 1) return ctx_fail(c, HOP_EINVAL, "offsets are required");
    const int64_t n = offsets[B];
    if (n <= 0 || n >= (int64_t(1) << 31) - 1) return ctx_fail(c, HOP_EINVAL, "bad total particle count");
    HOP_CUDA(c, cudaSetDevice(c->device));
    int32_t *group = nullptr;
    HOP_CUDA(c, cudaMalloc(&group, n * sizeof(int32_t)));
    std::vector<int64_t> ng(B);
    hop_tuning saved;
    hop_get_tuning(c, &saved);
    int rc = HOP_OK, pick = -1;
    float best_ms = 0.f;
    for (int i = 0; i < n_cand && rc == HOP_OK; ++i) {
        cand[i].ms = -1.f;
        if (cand[i].qpw != 4 && cand[i].qpw != 8 && cand[i].qpw != 16 && cand[i].qpw != 32) continue;
        if (hop_apply_tuning(c, &cand[i]) != HOP_OK) continue;
        if (p && p->radius_mode == HOP_RADIUS_LEARNED && !c->mlp->loaded) continue;
        // the first run captures the pass; the timed ones replay it
        rc = hop_run_batch(c, pos, offsets, boxes, B, p, nullptr, group, ng.data(), nullptr, 0, 0);
        std::vector<float> t;
        for (int r = 0; r < reps && rc == HOP_OK; ++r) {
            rc = hop_run_batch(c, pos, offsets, boxes, B, p, nullptr, group, ng.data(), nullptr, 0, 0);
            t.push_back((float)c->stats.ms_total);
        }
        if (rc) break;
        std::sort(t.begin(), t.end());
        cand[i].ms = t[t.size() / 2];
        if (pick < 0 || cand[i].ms < best_ms) {
            pick = i;
            best_ms = cand[i].ms;
        }
    }
    graph_drop(c);   // the cached graph writes to `group`
    cudaFree(group);
    if (rc) {
        hop_apply_tuning(c, &saved);
        return rc;
    }
    if (pick < 0) {
        hop_apply_tuning(c, &saved);
        return ctx_fail(c, HOP_EINVAL, "no candidate could run");
    }
    *best = pick;
    return hop_apply_tuning(c, &cand[pick]);
}

}  // extern "C"
