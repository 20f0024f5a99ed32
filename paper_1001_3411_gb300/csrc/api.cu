// C ABI of libhop (declared in include/hop.h): contexts, scratch memory,
// argument checks and the order in which each call runs the kernels.
#include "hop_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

// ------------------------------------------------------------ context ----
int ctx_fail(hop_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int ctx_cuda(hop_ctx *c, cudaError_t e, const char *what)
{
    if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? HOP_ENOMEM : HOP_ECUDA;
}

void *ctx_buf(hop_ctx *c, Slot s, size_t bytes)
{
    DevBuf &b = c->buf[s];
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return b.p;
    if (b.p) {
        if (c->capturing) {
            // nodes captured earlier use the old buffer: keep it with the graph
            c->graveyard.push_back(b.p);
        } else {
            // work already enqueued may still use the old buffer
            cudaStreamSynchronize(c->stream);
            cudaFree(b.p);
        }
        b.p = nullptr;
        b.cap = 0;
    }
    ++c->buf_epoch;   // a cached graph that used this slot is stale
    size_t want = bytes + bytes / 8;
    want = (want + (size_t(2) << 20) - 1) & ~((size_t(2) << 20) - 1);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&b.p, bytes);
        want = bytes;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        c->err = "device allocation of " + std::to_string(bytes) + " bytes failed";
        return nullptr;
    }
    b.cap = want;
    return b.p;
}

int ctx_check_device_error(hop_ctx *c)
{
    uint32_t *h = (uint32_t *)c->h_pinned;
    HOP_CUDA(c, cudaMemcpyAsync(h, c->d_err, 4, cudaMemcpyDeviceToHost, c->stream));
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    const uint32_t e = h[0];
    if (!e) return HOP_OK;
    HOP_CUDA(c, cudaMemsetAsync(c->d_err, 0, 4, c->stream));
    if (e & kErrBadPos) return ctx_fail(c, HOP_EINVAL, "a coordinate lies outside [0, box) or is NaN");
    if (e & kErrBadIndex) return ctx_fail(c, HOP_EINVAL, "an index array holds a value >= n");
    if (e & kErrDegenerate)
        return ctx_fail(c, HOP_EDEGENERATE, "more equidistant neighbours than the search buffer holds");
    if (e & kErrKnnRetry) return ctx_fail(c, HOP_ETIMEOUT, "kNN search did not certify");
    if (e & kErrChainLoop) return ctx_fail(c, HOP_ETIMEOUT, "chain following did not end");
    if (e & kErrMergeLoop) return ctx_fail(c, HOP_ETIMEOUT, "merge rounds did not converge");
    if (e & kErrTableFull) return ctx_fail(c, HOP_ENOMEM, "boundary table full");
    if (e & kErrChainCap) return ctx_fail(c, HOP_ENOMEM, "more chains than the merge arrays hold");
    if (e & kErrSortWait) return ctx_fail(c, HOP_ETIMEOUT, "a radix sort pass waited too long for an earlier tile");
    return ctx_fail(c, HOP_ECUDA, "device error word " + std::to_string(e));
}

namespace {

bool is_host_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

int check_params(hop_ctx *c, const hop_params *p, int64_t n)
{
    if (!p) return ctx_fail(c, HOP_EINVAL, "params is NULL");
    if (p->n_dens < 2 || p->n_dens > kMaxDens) return ctx_fail(c, HOP_EINVAL, "n_dens must be in [2, 128]");
    if (p->n_hop < 1 || p->n_hop > p->n_dens)
        return ctx_fail(c, HOP_EINVAL, "n_hop must be in [1, n_dens]");
    if (p->n_merge < 1 || p->n_merge > p->n_hop) return ctx_fail(c, HOP_EINVAL, "n_merge must be in [1, n_hop]");
    if (!(p->box > 0) || !std::isfinite(p->box)) return ctx_fail(c, HOP_EINVAL, "box must be positive");
    if (n < p->n_dens) return ctx_fail(c, HOP_EINVAL, "need at least n_dens particles");
    if (n >= (int64_t(1) << 31) - 1) return ctx_fail(c, HOP_EINVAL, "n must be < 2^31 - 1");
    if (p->radius_mode < HOP_RADIUS_PLAIN || p->radius_mode > HOP_RADIUS_LEARNED)
        return ctx_fail(c, HOP_EINVAL, "unknown radius_mode");
    return HOP_OK;
}


void ev_record(hop_ctx *c, int i) { cudaEventRecord(c->ev[i], c->stream); }

double ev_ms(hop_ctx *c, int a, int b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return ms;
}

struct DensityState {
    void *spos;
    uint32_t *perm;
    uint64_t *keys;
    uint32_t *cellT;
    int Ld;
    uint32_t *nbr_s;
    int ld_s;
    float *dens_s;
    float *rk_s;
};

// Grid build, first radii and the kNN + density pass, all in sorted order.
int density_core(hop_ctx *c, const void *pos, int64_t n, const hop_params *p, int n_out,
                 DensityState *st)
{
    HOP_CUDA(c, cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * 16, c->stream));
    ev_record(c, 0);
    int rc = grid_build(c, pos, n, p, &st->spos, &st->perm, &st->keys, &st->cellT, &st->Ld);
    if (rc) return rc;
    ev_record(c, 1);
    const int qpw = c->qpw;
    const int64_t n_chunks = (n + qpw - 1) / qpw;
    float *chunk_r = nullptr;
    if (p->radius_mode == HOP_RADIUS_COUNT) {
        chunk_r = (float *)ctx_buf(c, S_CHUNK_R, n_chunks * sizeof(float));
        if (!chunk_r) return HOP_ENOMEM;
        rc = chunk_radius(c, st->spos, st->keys, st->cellT, st->Ld, n, p, qpw, chunk_r);
        if (rc) return rc;
    } else if (p->radius_mode == HOP_RADIUS_LEARNED) {
        if (!c->mlp->loaded) return ctx_fail(c, HOP_ENOMODEL, "no radius network loaded (hop_mlp_load)");
        chunk_r = (float *)ctx_buf(c, S_CHUNK_R, n_chunks * sizeof(float));
        if (!chunk_r) return HOP_ENOMEM;
        rc = mlp_radius(c, st->spos, st->keys, st->cellT, st->Ld, n, p, qpw, chunk_r);
        if (rc) return rc;
    }
    ev_record(c, 2);
    st->ld_s = std::max(n_out, 1);
    st->nbr_s = n_out > 0 ? (uint32_t *)ctx_buf(c, S_NBR_S, (size_t)n * st->ld_s * sizeof(uint32_t)) : nullptr;
    st->dens_s = (float *)ctx_buf(c, S_DENS_S, n * sizeof(float));
    st->rk_s = (float *)ctx_buf(c, S_RK_S, n * sizeof(float));
    if ((n_out > 0 && !st->nbr_s) || !st->dens_s || !st->rk_s) return HOP_ENOMEM;
    KnnArgs a;
    a.spos = st->spos;
    a.keys = st->keys;
    a.cellT = st->cellT;
    a.level_dense = st->Ld;
    a.n = n;
    a.box = p->box;
    a.k = p->n_dens;
    a.n_out = n_out;
    a.ld_out = st->ld_s;
    a.chunk_r = chunk_r;
    a.plain_r = plain_radius_for(n, p->box, p->n_dens);
    a.n_norm = c->norm_n;
    a.nbr_s = st->nbr_s;
    a.dens_s = st->dens_s;
    a.rk_s = st->rk_s;
    rc = knn_launch(c, a, p->pos_is_f64 != 0, qpw, c->cpr);
    if (rc) return rc;
    ev_record(c, 3);
    c->last_n = n;
    c->last_level_dense = st->Ld;
    c->last_qpw = qpw;
    c->last_box = p->box;
    c->last_f64 = p->pos_is_f64 != 0;
    c->last_ndens = p->n_dens;
    c->last_spos = st->spos;
    c->last_keys = st->keys;
    c->last_cellT = st->cellT;
    c->last_rk = st->rk_s;
    return HOP_OK;
}

void read_counters(hop_ctx *c)
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

}  // namespace

// ------------------------------------------------------------ C ABI ------
extern "C" {

void hop_default_params(hop_params *p)
{
    if (!p) return;
    p->n_dens = 64;
    p->n_hop = 16;
    p->n_merge = 4;
    p->delta_outer = 80.f;
    p->delta_saddle = 200.f;
    p->delta_peak = 240.f;
    p->box = 1.0;
    p->pos_is_f64 = 0;
    p->radius_mode = HOP_RADIUS_PLAIN;
}

int hop_create(hop_ctx **out, int device, void *cuda_stream)
{
    if (!out) return HOP_EINVAL;
    *out = nullptr;
    hop_ctx *c = new (std::nothrow) hop_ctx();
    if (!c) return HOP_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    int rc = HOP_OK;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, 512);
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, 512);
    if (e == cudaSuccess) c->d_counters = (unsigned long long *)((char *)c->d_err + 256);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_pinned, 4096);
    for (int i = 0; e == cudaSuccess && i < 12; ++i) e = cudaEventCreate(&c->ev[i]);
    if (e != cudaSuccess) {
        rc = ctx_cuda(c, e, "hop_create");
        hop_destroy(c);
        return rc;
    }
    *out = c;
    return HOP_OK;
}

void hop_destroy(hop_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    batch_free(c);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (int i = 0; i < S_COUNT; ++i)
        if (c->buf[i].p) cudaFree(c->buf[i].p);
    if (c->d_err) cudaFree(c->d_err);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    for (int i = 0; i < 12; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    mlp_free(c);
    cudaGetLastError();
    delete c;
}

int hop_set_stream(hop_ctx *c, void *cuda_stream)
{
    if (!c) return HOP_EINVAL;
    c->stream = (cudaStream_t)cuda_stream;
    return HOP_OK;
}

const char *hop_last_error(const hop_ctx *c) { return c ? c->err.c_str() : "null context"; }

int hop_set_tuning(hop_ctx *c, int32_t qpw, int32_t cpr)
{
    if (!c) return HOP_EINVAL;
    if (qpw != 0 && qpw != 1 && qpw != 2 && qpw != 4 && qpw != 8 && qpw != 16 && qpw != 32)
        return ctx_fail(c, HOP_EINVAL, "queries per warp must be 1, 2, 4, 8, 16 or 32");
    if (cpr < 0 || cpr > 4) return ctx_fail(c, HOP_EINVAL, "cells per radius must be 1 to 4");
    if (qpw) {
        c->qpw = qpw;
        c->mlp = c->mlp_bank + qpw_index(qpw);
    }
    if (cpr) c->cpr = cpr;
    return HOP_OK;
}

int hop_density(hop_ctx *c, const void *pos, int64_t n, const hop_params *p, uint32_t *nbr,
                int32_t ld_nbr, float *dens, float *rk)
{
    if (!c) return HOP_EINVAL;
    c->err.clear();
    int rc = check_params(c, p, n);
    if (rc) return rc;
    if (!pos || !dens) return ctx_fail(c, HOP_EINVAL, "pos and dens are required");
    if (nbr && (ld_nbr < p->n_hop || ld_nbr > p->n_dens))
        return ctx_fail(c, HOP_EINVAL, "ld_nbr must be in [n_hop, n_dens]");
    HOP_CUDA(c, cudaSetDevice(c->device));
    const int64_t launches0 = c->launches;
    DensityState st;
    rc = density_core(c, pos, n, p, nbr ? ld_nbr : 0, &st);
    if (rc) return rc;
    rc = ctx_check_device_error(c);   // lists of an uncertified search are not valid indices
    if (rc) return rc;
    rc = scatter_outputs(c, st.perm, n, st.dens_s, dens, nullptr, nullptr, st.nbr_s, st.ld_s, nbr,
                         ld_nbr, nbr ? ld_nbr : 0, nullptr, nullptr);
    if (rc) return rc;
    if (rk) {
        rc = scatter_outputs(c, st.perm, n, st.rk_s, rk, nullptr, nullptr, nullptr, 0, nullptr, 0, 0,
                             nullptr, nullptr);
        if (rc) return rc;
    }
    ev_record(c, 4);
    rc = ctx_check_device_error(c);
    read_counters(c);
    c->stats.ms_sort = ev_ms(c, 0, 1);
    c->stats.ms_radius = ev_ms(c, 1, 2);
    c->stats.ms_knn = ev_ms(c, 2, 3);
    c->stats.ms_total = ev_ms(c, 0, 4);
    c->stats.launches = c->launches - launches0;
    return rc;
}

int hop_link(hop_ctx *c, const float *dens, const uint32_t *nbr, int32_t ld_nbr, int64_t n,
             int32_t n_hop, uint32_t *hop, uint32_t *chain)
{
    if (!c) return HOP_EINVAL;
    c->err.clear();
    if (!dens || !nbr || !chain || n <= 0) return ctx_fail(c, HOP_EINVAL, "dens, nbr, chain and n > 0 are required");
    if (n_hop < 1 || n_hop > ld_nbr) return ctx_fail(c, HOP_EINVAL, "n_hop must be in [1, ld_nbr]");
    HOP_CUDA(c, cudaSetDevice(c->device));
    uint64_t *dkey = (uint64_t *)ctx_buf(c, S_DKEY, n * sizeof(uint64_t));
    if (!dkey) return HOP_ENOMEM;
    int rc = make_dkey(c, dens, nullptr, n, dkey);
    if (rc) return rc;
    return hop_links(c, dkey, nbr, ld_nbr, n, n_hop, hop, chain);
}

// Writes m table entries (ek, es) to the caller's arrays in ascending pair
// order.  Synchronises the stream.
static int write_sorted_edges(hop_ctx *c, const uint64_t *ek, const double *es, int64_t m, uint64_t *edge_pair,
                              double *edge_sum)
{
    if (m == 0) return HOP_OK;
    uint64_t *k1 = (uint64_t *)ctx_buf(c, S_ESORT_K0, m * sizeof(uint64_t));
    uint64_t *k2 = (uint64_t *)ctx_buf(c, S_ESORT_K1, m * sizeof(uint64_t));
    uint32_t *v1 = (uint32_t *)ctx_buf(c, S_ESORT_V0, m * sizeof(uint32_t));
    uint32_t *v2 = (uint32_t *)ctx_buf(c, S_ESORT_V1, m * sizeof(uint32_t));
    void *tmp = ctx_buf(c, S_ESORT_TMP, radix_sort_scratch_bytes(m));
    if (!k1 || !k2 || !v1 || !v2 || !tmp) return HOP_ENOMEM;
    HOP_CUDA(c, cudaMemcpyAsync(k1, ek, m * sizeof(uint64_t), cudaMemcpyDeviceToDevice, c->stream));
    int rc = iota_u32(c, v1, m);
    if (rc) return rc;
    rc = radix_sort_u64(c, k1, k2, v1, v2, m, 0, 64, tmp);
    if (rc) return rc;
    HOP_CUDA(c, cudaMemcpyAsync(edge_pair, k1, m * sizeof(uint64_t), cudaMemcpyDeviceToDevice, c->stream));
    // the sums, in the same order
    rc = gather_f64(c, es, v1, m, edge_sum);
    if (rc) return rc;
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    return HOP_OK;
}

int hop_boundaries(hop_ctx *c, const uint32_t *chain, const float *dens, const uint32_t *nbr,
                   int32_t ld_nbr, int64_t n, int32_t n_merge, float delta_outer,
                   uint64_t *edge_pair, double *edge_sum, int64_t cap, int64_t *n_edges)
{
    if (!c) return HOP_EINVAL;
    c->err.clear();
    if (!chain || !dens || !nbr || !n_edges || n <= 0) return ctx_fail(c, HOP_EINVAL, "missing argument");
    if (n_merge < 1 || n_merge > ld_nbr) return ctx_fail(c, HOP_EINVAL, "n_merge must be in [1, ld_nbr]");
    HOP_CUDA(c, cudaSetDevice(c->device));
    uint64_t *dkey = (uint64_t *)ctx_buf(c, S_DKEY, n * sizeof(uint64_t));
    if (!dkey) return HOP_ENOMEM;
    int rc = make_dkey(c, dens, nullptr, n, dkey);
    if (rc) return rc;
    uint64_t *ek;
    double *es;
    int64_t m;
    rc = boundaries_table(c, chain, dkey, nbr, ld_nbr, n, n_merge, delta_outer, &ek, &es, &m);
    if (rc) return rc;
    *n_edges = m;
    if (m > cap || !edge_pair || !edge_sum) {
        if (m > cap) return ctx_fail(c, HOP_ETABLE, "edge capacity too small");
        return ctx_fail(c, HOP_EINVAL, "edge_pair and edge_sum are required");
    }
    return write_sorted_edges(c, ek, es, m, edge_pair, edge_sum);
}

int hop_boundaries_reduce(hop_ctx *c, const uint64_t *pair_in, const double *sum_in, int64_t m_in,
                          uint64_t *edge_pair, double *edge_sum, int64_t cap, int64_t *n_edges)
{
    if (!c) return HOP_EINVAL;
    c->err.clear();
    if (!n_edges || m_in < 0 || (m_in > 0 && (!pair_in || !sum_in))) return ctx_fail(c, HOP_EINVAL, "missing argument");
    HOP_CUDA(c, cudaSetDevice(c->device));
    uint64_t *ek;
    double *es;
    int64_t m;
    int rc = edges_max_table(c, pair_in, sum_in, m_in, &ek, &es, &m);
    if (rc) return rc;
    *n_edges = m;
    if (m > cap || (m > 0 && (!edge_pair || !edge_sum))) {
        if (m > cap) return ctx_fail(c, HOP_ETABLE, "edge capacity too small");
        return ctx_fail(c, HOP_EINVAL, "edge_pair and edge_sum are required");
    }
    return write_sorted_edges(c, ek, es, m, edge_pair, edge_sum);
}

int hop_set_norm_count(hop_ctx *c, int64_t n_norm)
{
    if (!c) return HOP_EINVAL;
    if (n_norm < 0) return ctx_fail(c, HOP_EINVAL, "the normalisation count must be >= 0");
    c->norm_n = n_norm;
    return HOP_OK;
}

int hop_merge(hop_ctx *c, const uint32_t *chain, const float *dens, int64_t n,
              const uint64_t *edge_pair, const double *edge_sum, int64_t n_edges,
              float delta_outer, float delta_saddle, float delta_peak, int32_t *group,
              int64_t *n_groups)
{
    if (!c) return HOP_EINVAL;
    c->err.clear();
    if (!chain || !dens || !group || !n_groups || n <= 0 || n_edges < 0 ||
        (n_edges > 0 && (!edge_pair || !edge_sum)))
        return ctx_fail(c, HOP_EINVAL, "missing argument");
    HOP_CUDA(c, cudaSetDevice(c->device));
    uint64_t *dkey = (uint64_t *)ctx_buf(c, S_DKEY, n * sizeof(uint64_t));
    if (!dkey) return HOP_ENOMEM;
    int rc = make_dkey(c, dens, nullptr, n, dkey);
    if (rc) return rc;
    rc = merge_groups(c, chain, dkey, n, edge_pair, edge_sum, n_edges, delta_outer, delta_saddle,
                      delta_peak, group, n_groups);
    if (rc) return rc;
    return ctx_check_device_error(c);
}

int hop_run(hop_ctx *c, const void *pos, int64_t n, const hop_params *p, float *dens,
            int32_t *group, int64_t *n_groups, uint32_t *nbr, int32_t ld_nbr, uint32_t *chain)
{
    if (!c) return HOP_EINVAL;
    c->err.clear();
    int rc = check_params(c, p, n);
    if (rc) return rc;
    if (!pos || !group || !n_groups) return ctx_fail(c, HOP_EINVAL, "pos, group and n_groups are required");
    if (nbr && (ld_nbr < p->n_hop || ld_nbr > p->n_dens))
        return ctx_fail(c, HOP_EINVAL, "ld_nbr must be in [n_hop, n_dens]");
    HOP_CUDA(c, cudaSetDevice(c->device));
    const size_t pos_bytes = (size_t)n * 3 * (p->pos_is_f64 ? 8 : 4);
    const bool host_pos = is_host_ptr(pos);
    const bool host_dens = dens && is_host_ptr(dens);
    const bool host_group = is_host_ptr(group);
    const int64_t launches0 = c->launches;
    ev_record(c, 8);
    const void *dpos = pos;
    if (host_pos) {
        void *b = ctx_buf(c, S_POS_IN, pos_bytes);
        if (!b) return HOP_ENOMEM;
        HOP_CUDA(c, cudaMemcpyAsync(b, pos, pos_bytes, cudaMemcpyHostToDevice, c->stream));
        dpos = b;
    }
    DensityState st;
    const int n_out = std::max<int>(p->n_hop, nbr ? ld_nbr : 0);
    rc = density_core(c, dpos, n, p, n_out, &st);
    if (rc) return rc;
    rc = ctx_check_device_error(c);
    if (rc) return rc;
    // link in sorted order
    uint64_t *dkey = (uint64_t *)ctx_buf(c, S_DKEY, n * sizeof(uint64_t));
    uint32_t *hop_s = (uint32_t *)ctx_buf(c, S_HOP, n * sizeof(uint32_t));
    uint32_t *chain_s = (uint32_t *)ctx_buf(c, S_CHAIN, n * sizeof(uint32_t));
    if (!dkey || !hop_s || !chain_s) return HOP_ENOMEM;
    rc = make_dkey(c, st.dens_s, st.perm, n, dkey);
    if (rc) return rc;
    rc = hop_links(c, dkey, st.nbr_s, st.ld_s, n, p->n_hop, hop_s, chain_s);
    if (rc) return rc;
    ev_record(c, 5);
    uint64_t *ek;
    double *es;
    int64_t m;
    rc = boundaries_table(c, chain_s, dkey, st.nbr_s, st.ld_s, n, p->n_merge, p->delta_outer, &ek, &es, &m);
    if (rc) return rc;
    ev_record(c, 6);
    int32_t *group_s = (int32_t *)ctx_buf(c, S_GROUP_OUT, n * sizeof(int32_t));
    if (!group_s) return HOP_ENOMEM;
    rc = merge_groups(c, chain_s, dkey, n, ek, es, m, p->delta_outer, p->delta_saddle, p->delta_peak,
                      group_s, n_groups);
    if (rc) return rc;
    ev_record(c, 7);
    // results in the caller's order
    float *dens_dev = dens;
    int32_t *group_dev = group;
    if (host_dens || host_group) {
        if (host_dens) dens_dev = (float *)ctx_buf(c, S_OUT_DENS, n * sizeof(float));
        if (host_group) group_dev = (int32_t *)ctx_buf(c, S_OUT_GROUP, n * sizeof(int32_t));
        if ((host_dens && !dens_dev) || (host_group && !group_dev)) return HOP_ENOMEM;
    }
    rc = scatter_outputs(c, st.perm, n, st.dens_s, dens_dev, group_s, group_dev, st.nbr_s, st.ld_s,
                         nbr, ld_nbr, nbr ? ld_nbr : 0, chain ? chain_s : nullptr, chain);
    if (rc) return rc;
    if (host_dens)
        HOP_CUDA(c, cudaMemcpyAsync(dens, dens_dev, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (host_group)
        HOP_CUDA(c, cudaMemcpyAsync(group, group_dev, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    ev_record(c, 9);
    rc = ctx_check_device_error(c);
    read_counters(c);
    c->stats.ms_sort = ev_ms(c, 0, 1);
    c->stats.ms_radius = ev_ms(c, 1, 2);
    c->stats.ms_knn = ev_ms(c, 2, 3);
    c->stats.ms_link = ev_ms(c, 3, 5);
    c->stats.ms_boundaries = ev_ms(c, 5, 6);
    c->stats.ms_merge = ev_ms(c, 6, 7);
    c->stats.ms_total = ev_ms(c, 8, 9);
    c->stats.launches = c->launches - launches0;
    return rc;
}

int hop_get_stats(const hop_ctx *c, hop_stats *out)
{
    if (!c || !out) return HOP_EINVAL;
    *out = c->stats;
    return HOP_OK;
}

}  // extern "C"
