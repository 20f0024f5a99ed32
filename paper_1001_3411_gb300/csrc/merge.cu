// HOP merging steps 1, 2, 4, 5 (Parallel HOP Sec. 2, Fig. 1) on the GPU.
//
//  M1  chains = roots (chain[i] == i) with density >= delta_outer, numbered
//      densely by a scan; every boundary endpoint is such a root.
//  M2  proto-halos: root density >= delta_peak.
//  M3  edges sorted once in the strict merge order (s desc, lo asc, hi asc,
//      lo/hi the roots' original indices) by two stable radix sorts, so an
//      edge's position is its rank.
//  M4  proto-halos joined by a direct boundary s >= 2 delta_saddle:
//      connected components (hook to the smaller root + compress, until no
//      edge joins two roots).  Each component is an owned set.
//  M5  sub-peak chains: Boruvka rounds on the maximum spanning forest of the
//      boundary graph with all owned sets contracted.  In a round every
//      unowned component picks its best edge (smallest rank) to another
//      component not both owned; it hooks to the other side (owned targets
//      absorb it; a mutual pick keeps the smaller label as root).  Owned sets
//      never pick, so no two owned sets meet.  Under a strict edge order the
//      forest is unique, hence equal to the sequential Kruskal reading.
//  M6  groups = owned sets, ranked by their peak key (density desc, index
//      asc); group per particle with the delta_outer cut.
#include "hop_internal.cuh"

#include <algorithm>

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kMaxRounds = 64;

__global__ void root_flag_kernel(const uint32_t *__restrict__ chain, const uint64_t *__restrict__ dkey,
                                 int64_t n, float d_o, uint32_t *__restrict__ flag,
                                 uint32_t *__restrict__ err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = chain[i];
        if (c >= (uint64_t)n || chain[c] != c) atomicOr(err, kErrBadIndex);
        flag[i] = (c == (uint32_t)i && key_dens(dkey[i]) >= d_o) ? 1u : 0u;
    }
}

__global__ void root_list_kernel(const uint32_t *__restrict__ chain, const uint64_t *__restrict__ dkey,
                                 int64_t n, float d_o, float d_p, const uint32_t *__restrict__ cid,
                                 uint64_t *__restrict__ ckey, uint8_t *__restrict__ own, int64_t c_cap,
                                 uint32_t *__restrict__ err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (chain[i] != (uint32_t)i) continue;
        const uint64_t k = dkey[i];
        if (!(key_dens(k) >= d_o)) continue;
        const uint32_t c = cid[i];
        if (c >= (uint64_t)c_cap) {
            atomicOr(err, kErrChainCap);
            continue;
        }
        ckey[c] = k;
        own[c] = key_dens(k) >= d_p ? 1 : 0;
    }
}

// Edge endpoints -> dense chain ids; sort key for (lo_orig, hi_orig).
__global__ void edge_prep_kernel(const uint64_t *__restrict__ ekey, const double *__restrict__ esum,
                                 DevCount mc, int64_t n, const uint32_t *__restrict__ chain,
                                 const uint32_t *__restrict__ cid, const uint64_t *__restrict__ dkey,
                                 float d_o, uint32_t *__restrict__ ea, uint32_t *__restrict__ eb,
                                 uint64_t *__restrict__ k1, uint32_t *__restrict__ v1,
                                 uint32_t *__restrict__ err, int64_t c_cap)
{
    const int64_t m = mc.get();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t lo = (uint32_t)(ekey[e] >> 32), hi = (uint32_t)ekey[e];
        const bool bad = lo >= (uint64_t)n || hi >= (uint64_t)n || chain[lo] != lo || chain[hi] != hi ||
                         !(key_dens(dkey[lo]) >= d_o) || !(key_dens(dkey[hi]) >= d_o) || lo == hi;
        if (bad || cid[lo] >= (uint64_t)c_cap || cid[hi] >= (uint64_t)c_cap) {
            atomicOr(err, bad ? kErrBadIndex : kErrChainCap);
            ea[e] = eb[e] = 0;
            k1[e] = 0;
            v1[e] = (uint32_t)e;
            continue;
        }
        const uint32_t olo = key_orig(dkey[lo]), ohi = key_orig(dkey[hi]);
        ea[e] = cid[lo];
        eb[e] = cid[hi];
        k1[e] = olo < ohi ? (((uint64_t)olo << 32) | ohi) : (((uint64_t)ohi << 32) | olo);
        v1[e] = (uint32_t)e;
        (void)esum;
    }
}

__global__ void edge_key2_kernel(const double *__restrict__ esum, const uint32_t *__restrict__ order,
                                 DevCount mc, uint64_t *__restrict__ k2)
{
    const int64_t m = mc.get();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x)
        k2[t] = ~(uint64_t)__double_as_longlong(esum[order[t]]);
}

__global__ void edge_permute_kernel(const uint32_t *__restrict__ order, DevCount mc,
                                    const uint32_t *__restrict__ ea, const uint32_t *__restrict__ eb,
                                    const double *__restrict__ esum, uint32_t *__restrict__ sa,
                                    uint32_t *__restrict__ sb, double *__restrict__ ss)
{
    const int64_t m = mc.get();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = order[t];
        sa[t] = ea[e];
        sb[t] = eb[e];
        ss[t] = esum[e];
    }
}

__global__ void iota_kernel(uint32_t *p, DevCount nc)
{
    const int64_t n = nc.get();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (uint32_t)i;
}

__global__ void fill_kernel(uint32_t *p, DevCount nc, uint32_t v)
{
    const int64_t n = nc.get();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void proto_hook_kernel(const uint32_t *__restrict__ sa, const uint32_t *__restrict__ sb,
                                  const double *__restrict__ ss, DevCount mc, double two_ds,
                                  const uint8_t *__restrict__ own, uint32_t *parent,
                                  uint32_t *changed)
{
    const int64_t m = mc.get();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = sa[t], b = sb[t];
        if (!own[a] || !own[b] || !(ss[t] >= two_ds)) continue;
        const uint32_t ra = find_root(parent, a), rb = find_root(parent, b);
        if (ra == rb) continue;
        atomicMin(&parent[max(ra, rb)], min(ra, rb));
        *changed = 1u;
    }
}

__global__ void compress_kernel(uint32_t *parent, DevCount cc)
{
    const int64_t C = cc.get();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x)
        parent[c] = find_root(parent, (uint32_t)c);
}

// Boruvka: every unowned component's smallest-rank eligible edge.
__global__ void best_edge_kernel(const uint32_t *__restrict__ sa, const uint32_t *__restrict__ sb,
                                 DevCount mc, const uint32_t *__restrict__ parent,
                                 const uint8_t *__restrict__ own, uint32_t *__restrict__ best)
{
    const int64_t m = mc.get();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t ca = parent[sa[t]], cb = parent[sb[t]];
        if (ca == cb) continue;
        const bool oa = own[ca], ob = own[cb];
        if (oa && ob) continue;
        if (!oa) atomicMin(&best[ca], (uint32_t)t);
        if (!ob) atomicMin(&best[cb], (uint32_t)t);
    }
}

__global__ void target_kernel(const uint32_t *__restrict__ sa, const uint32_t *__restrict__ sb,
                              DevCount cc, const uint32_t *__restrict__ parent,
                              const uint8_t *__restrict__ own, const uint32_t *__restrict__ best,
                              uint32_t *__restrict__ tgt)
{
    const int64_t C = cc.get();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < C;
         x += (int64_t)gridDim.x * blockDim.x) {
        uint32_t y = kNone;
        if (parent[x] == (uint32_t)x && !own[x] && best[x] != kNone) {
            const uint32_t t = best[x];
            const uint32_t ca = parent[sa[t]], cb = parent[sb[t]];
            y = ca == (uint32_t)x ? cb : ca;
        }
        tgt[x] = y;
    }
}

__global__ void hook_kernel(DevCount cc, const uint8_t *__restrict__ own,
                            const uint32_t *__restrict__ best, const uint32_t *__restrict__ tgt,
                            uint32_t *parent, uint32_t *changed)
{
    const int64_t C = cc.get();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < C;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t y = tgt[x];
        if (y == kNone) continue;
        if (!own[y] && best[y] == best[x] && (uint32_t)x < y) continue;  // mutual: smaller stays root
        parent[x] = y;
        *changed = 1u;
    }
}

__global__ void group_peak_kernel(DevCount cc, const uint32_t *__restrict__ parent,
                                  const uint8_t *__restrict__ own, const uint64_t *__restrict__ ckey,
                                  unsigned long long *__restrict__ gpeak)
{
    const int64_t C = cc.get();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = parent[c];
        if (own[r]) atomicMax(&gpeak[r], (unsigned long long)ckey[c]);
    }
}

__global__ void group_flag_kernel(DevCount cc, const uint32_t *__restrict__ parent,
                                  const uint8_t *__restrict__ own, uint32_t *__restrict__ flag)
{
    const int64_t C = cc.get();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x)
        flag[c] = (parent[c] == (uint32_t)c && own[c]) ? 1u : 0u;
}

__global__ void group_list_kernel(DevCount cc, const uint32_t *__restrict__ flag,
                                  const uint32_t *__restrict__ pos,
                                  const unsigned long long *__restrict__ gpeak,
                                  uint64_t *__restrict__ gk, uint32_t *__restrict__ gv)
{
    const int64_t C = cc.get();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[c]) continue;
        gk[pos[c]] = ~(uint64_t)gpeak[c];
        gv[pos[c]] = (uint32_t)c;
    }
}

__global__ void group_rank_kernel(DevCount gc, const uint32_t *__restrict__ gv, uint32_t *__restrict__ grank)
{
    const int64_t G = gc.get();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x)
        grank[gv[g]] = (uint32_t)g;
}

__global__ void particle_group_kernel(const uint32_t *__restrict__ chain,
                                      const uint64_t *__restrict__ dkey, int64_t n, float d_o,
                                      const uint32_t *__restrict__ cid, DevCount cc,
                                      const uint32_t *__restrict__ parent,
                                      const uint8_t *__restrict__ own,
                                      const uint32_t *__restrict__ grank, int32_t *__restrict__ group,
                                      uint32_t *__restrict__ err)
{
    const int64_t C = cc.get();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = -1;
        if (key_dens(dkey[i]) >= d_o) {
            const uint32_t root = chain[i];
            // a member above delta_outer has a root above it (hops go uphill)
            if (!(key_dens(dkey[root]) >= d_o) || cid[root] >= (uint64_t)C) {
                atomicOr(err, kErrBadIndex);
            } else {
                const uint32_t r = parent[cid[root]];
                if (own[r]) g = (int32_t)grank[r];
            }
        }
        group[i] = g;
    }
}

// Batched pass: each group's subvolume (from its peak's original index) as
// a sort key, and the count of groups per subvolume.
__global__ void group_seg_kernel(DevCount gc, const uint32_t *__restrict__ gv,
                                 const uint64_t *__restrict__ ckey, const SegDesc *__restrict__ seg,
                                 int B, uint64_t *__restrict__ gsub, uint32_t *__restrict__ per_seg)
{
    const int64_t G = gc.get();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < G;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = seg_of_index(seg, B, (int64_t)key_orig(ckey[gv[t]]));
        gsub[t] = (uint64_t)b;
        atomicAdd(&per_seg[b], 1u);
    }
}

// Rank within the subvolume: position in (subvolume, peak key) order minus
// the subvolume's first position.
__global__ void group_rank_seg_kernel(DevCount gc, const uint32_t *__restrict__ gv,
                                      const uint64_t *__restrict__ gsub,
                                      const uint32_t *__restrict__ seg_start, uint32_t *__restrict__ grank)
{
    const int64_t G = gc.get();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < G;
         t += (int64_t)gridDim.x * blockDim.x)
        grank[gv[t]] = (uint32_t)t - seg_start[gsub[t]];
}

__global__ void fill_u64_n_kernel(unsigned long long *p, DevCount nc, unsigned long long v)
{
    const int64_t n = nc.get();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace

int merge_groups(hop_ctx *c, const uint32_t *chain, const uint64_t *dkey, int64_t n,
                 const uint64_t *edge_key, const double *edge_sum, int64_t m, float d_o, float d_s,
                 float d_p, int32_t *group, int64_t *n_groups)
{
    uint32_t *hp = (uint32_t *)c->h_pinned;
    uint32_t *misc = (uint32_t *)ctx_buf(c, S_MISC, 256);
    uint32_t *cid = (uint32_t *)ctx_buf(c, S_GROUP_S, (n + 1) * sizeof(uint32_t));
    if (!misc || !cid) return HOP_ENOMEM;
    uint32_t *d_total = misc, *d_changed = misc + 1, *d_merr = misc + 2;
    HOP_CUDA(c, cudaMemsetAsync(misc, 0, 16, c->stream));
    // M1
    root_flag_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, dkey, n, d_o, cid, d_merr);
    HOP_LAUNCH(c);
    int rc = scan_exclusive_u32(c, cid, cid, n, d_total);
    if (rc) return rc;
    HOP_CUDA(c, cudaMemcpyAsync(hp, misc, 12, cudaMemcpyDeviceToHost, c->stream));
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hp[2] & kErrBadIndex) return ctx_fail(c, HOP_EINVAL, "chain labels are not roots of [0, n)");
    const int64_t C = hp[0];
    c->stats.n_chains = C;
    c->stats.n_edges = m;
    // arrays over chains and edges
    const int64_t Cp = std::max<int64_t>(C, 1), mp = std::max<int64_t>(m, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t o_ckey = take(Cp * 8), o_own = take(Cp), o_parent = take(Cp * 4),
                 o_best = take(Cp * 4), o_tgt = take(Cp * 4), o_gpeak = take(Cp * 8),
                 o_flag = take((Cp + 1) * 4), o_grank = take(Cp * 4), o_ea = take(mp * 4),
                 o_eb = take(mp * 4), o_sa = take(mp * 4), o_sb = take(mp * 4), o_ss = take(mp * 8),
                 o_k1 = take(mp * 8), o_k1b = take(mp * 8), o_v1 = take(mp * 4),
                 o_v1b = take(mp * 4), o_gk = take(Cp * 8), o_gkb = take(Cp * 8),
                 o_gv = take(Cp * 4), o_gvb = take(Cp * 4);
    const size_t sort_tmp = std::max(radix_sort_scratch_bytes(mp), radix_sort_scratch_bytes(Cp));
    const size_t o_tmp = take(sort_tmp);
    char *base = (char *)ctx_buf(c, S_MERGE, off);
    if (!base) return HOP_ENOMEM;
    uint64_t *ckey = (uint64_t *)(base + o_ckey);
    uint8_t *own = (uint8_t *)(base + o_own);
    uint32_t *parent = (uint32_t *)(base + o_parent), *best = (uint32_t *)(base + o_best),
             *tgt = (uint32_t *)(base + o_tgt), *flag = (uint32_t *)(base + o_flag),
             *grank = (uint32_t *)(base + o_grank);
    unsigned long long *gpeak = (unsigned long long *)(base + o_gpeak);
    uint32_t *ea = (uint32_t *)(base + o_ea), *eb = (uint32_t *)(base + o_eb),
             *sa = (uint32_t *)(base + o_sa), *sb = (uint32_t *)(base + o_sb);
    double *ss = (double *)(base + o_ss);
    uint64_t *k1 = (uint64_t *)(base + o_k1), *k1b = (uint64_t *)(base + o_k1b);
    uint32_t *v1 = (uint32_t *)(base + o_v1), *v1b = (uint32_t *)(base + o_v1b);
    uint64_t *gk = (uint64_t *)(base + o_gk), *gkb = (uint64_t *)(base + o_gkb);
    uint32_t *gv = (uint32_t *)(base + o_gv), *gvb = (uint32_t *)(base + o_gvb);
    void *tmp = base + o_tmp;

    HOP_CUDA(c, cudaMemsetAsync(own, 0, Cp, c->stream));
    root_list_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, dkey, n, d_o, d_p, cid, ckey, own, Cp,
                                                            d_merr);
    HOP_LAUNCH(c);
    // M3: strict order
    if (m > 0) {
        edge_prep_kernel<<<grid_for(c, m), 256, 0, c->stream>>>(edge_key, edge_sum, DevCount{m, nullptr}, n, chain, cid,
                                                               dkey, d_o, ea, eb, k1, v1, d_merr, Cp);
        HOP_LAUNCH(c);
        rc = radix_sort_u64(c, k1, k1b, v1, v1b, m, 0, 64, tmp);
        if (rc) return rc;
        edge_key2_kernel<<<grid_for(c, m), 256, 0, c->stream>>>(edge_sum, v1, DevCount{m, nullptr}, k1);
        HOP_LAUNCH(c);
        rc = radix_sort_u64(c, k1, k1b, v1, v1b, m, 0, 64, tmp);
        if (rc) return rc;
        edge_permute_kernel<<<grid_for(c, m), 256, 0, c->stream>>>(v1, DevCount{m, nullptr}, ea, eb, edge_sum, sa, sb, ss);
        HOP_LAUNCH(c);
    }
    // M4: proto-halo components
    iota_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(parent, DevCount{C, nullptr});
    HOP_LAUNCH(c);
    int rounds = 0;
    for (; m > 0 && rounds < kMaxRounds; ++rounds) {
        HOP_CUDA(c, cudaMemsetAsync(d_changed, 0, 4, c->stream));
        proto_hook_kernel<<<grid_for(c, m), 256, 0, c->stream>>>(sa, sb, ss, DevCount{m, nullptr}, 2.0 * (double)d_s, own,
                                                                parent, d_changed);
        HOP_LAUNCH(c);
        compress_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(parent, DevCount{C, nullptr});
        HOP_LAUNCH(c);
        HOP_CUDA(c, cudaMemcpyAsync(hp, misc, 12, cudaMemcpyDeviceToHost, c->stream));
        HOP_CUDA(c, cudaStreamSynchronize(c->stream));
        if (hp[2] & kErrBadIndex) return ctx_fail(c, HOP_EINVAL, "boundary pair is not a pair of chains above delta_outer");
        if (!hp[1]) break;
    }
    if (rounds >= kMaxRounds) return ctx_fail(c, HOP_ETIMEOUT, "proto-halo merge did not converge");
    // M5: Boruvka over sub-peak chains
    for (rounds = 0; m > 0 && rounds < kMaxRounds; ++rounds) {
        HOP_CUDA(c, cudaMemsetAsync(d_changed, 0, 4, c->stream));
        fill_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(best, DevCount{C, nullptr}, kNone);
        HOP_LAUNCH(c);
        best_edge_kernel<<<grid_for(c, m), 256, 0, c->stream>>>(sa, sb, DevCount{m, nullptr}, parent, own, best);
        HOP_LAUNCH(c);
        target_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(sa, sb, DevCount{C, nullptr}, parent, own, best, tgt);
        HOP_LAUNCH(c);
        hook_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(DevCount{C, nullptr}, own, best, tgt, parent, d_changed);
        HOP_LAUNCH(c);
        compress_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(parent, DevCount{C, nullptr});
        HOP_LAUNCH(c);
        HOP_CUDA(c, cudaMemcpyAsync(hp, misc, 8, cudaMemcpyDeviceToHost, c->stream));
        HOP_CUDA(c, cudaStreamSynchronize(c->stream));
        if (!hp[1]) break;
    }
    if (rounds >= kMaxRounds) return ctx_fail(c, HOP_ETIMEOUT, "sub-peak merge did not converge");
    // owned status of a root is its own (owned sets never hook); M6: groups
    HOP_CUDA(c, cudaMemsetAsync(gpeak, 0, Cp * 8, c->stream));
    group_peak_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(DevCount{C, nullptr}, parent, own, ckey, gpeak);
    HOP_LAUNCH(c);
    group_flag_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(DevCount{C, nullptr}, parent, own, flag);
    HOP_LAUNCH(c);
    uint32_t *gpos = tgt;   // reuse
    rc = scan_exclusive_u32(c, flag, gpos, C, d_total);
    if (rc) return rc;
    HOP_CUDA(c, cudaMemcpyAsync(hp, misc, 4, cudaMemcpyDeviceToHost, c->stream));
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    const int64_t G = C > 0 ? hp[0] : 0;
    if (G > 0) {
        group_list_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(DevCount{C, nullptr}, flag, gpos, gpeak, gk, gv);
        HOP_LAUNCH(c);
        rc = radix_sort_u64(c, gk, gkb, gv, gvb, G, 0, 64, tmp);
        if (rc) return rc;
        group_rank_kernel<<<grid_for(c, G), 256, 0, c->stream>>>(DevCount{G, nullptr}, gv, grank);
        HOP_LAUNCH(c);
    }
    particle_group_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, dkey, n, d_o, cid, DevCount{C, nullptr}, parent,
                                                                own, grank, group, c->d_err);
    HOP_LAUNCH(c);
    *n_groups = G;
    c->stats.n_groups = G;
    return HOP_OK;
}

// ------------------------------------------------------------ batched ----
// The same steps with every data-dependent size (chains, edges, groups) kept
// on the device, so the whole pass can be captured into one CUDA graph.
// Arrays are sized by their bounds (chains <= n, edges <= table capacity);
// kernels read the true counts.  Merge rounds are device-bounded loops.
namespace {

struct RoundArgs {
    const uint32_t *sa, *sb;
    const double *ss;
    DevCount m, C;
    double two_ds;
    const uint8_t *own;
    uint32_t *parent, *best, *tgt, *changed;
    int64_t cmax, mmax;
};

int proto_round(hop_ctx *c, void *p)
{
    const RoundArgs &r = *(const RoundArgs *)p;
    proto_hook_kernel<<<grid_for(c, r.mmax), 256, 0, c->stream>>>(r.sa, r.sb, r.ss, r.m, r.two_ds, r.own,
                                                                  r.parent, r.changed);
    HOP_LAUNCH(c);
    compress_kernel<<<grid_for(c, r.cmax), 256, 0, c->stream>>>(r.parent, r.C);
    HOP_LAUNCH(c);
    return HOP_OK;
}

int boruvka_round(hop_ctx *c, void *p)
{
    const RoundArgs &r = *(const RoundArgs *)p;
    fill_kernel<<<grid_for(c, r.cmax), 256, 0, c->stream>>>(r.best, r.C, kNone);
    HOP_LAUNCH(c);
    best_edge_kernel<<<grid_for(c, r.mmax), 256, 0, c->stream>>>(r.sa, r.sb, r.m, r.parent, r.own, r.best);
    HOP_LAUNCH(c);
    target_kernel<<<grid_for(c, r.cmax), 256, 0, c->stream>>>(r.sa, r.sb, r.C, r.parent, r.own, r.best, r.tgt);
    HOP_LAUNCH(c);
    hook_kernel<<<grid_for(c, r.cmax), 256, 0, c->stream>>>(r.C, r.own, r.best, r.tgt, r.parent, r.changed);
    HOP_LAUNCH(c);
    compress_kernel<<<grid_for(c, r.cmax), 256, 0, c->stream>>>(r.parent, r.C);
    HOP_LAUNCH(c);
    return HOP_OK;
}

}  // namespace

int merge_groups_graph(hop_ctx *c, const MergeGraphArgs &a)
{
    const int64_t n = a.n, mmax = std::max<int64_t>(a.m.max, 1);
    const int64_t Cmax = std::max<int64_t>(a.c_cap > 0 && a.c_cap < n ? a.c_cap : n, 1);
    uint32_t *d_C = a.counts, *d_G = a.counts + 1, *d_changed = a.counts + 2;
    uint32_t *d_round1 = a.counts + 3, *d_round2 = a.counts + 4;
    const DevCount C{Cmax, d_C}, G{Cmax, d_G};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t o_cid = take((n + 1) * 4), o_ckey = take(Cmax * 8), o_own = take(Cmax),
                 o_parent = take(Cmax * 4), o_best = take(Cmax * 4), o_tgt = take(Cmax * 4),
                 o_gpeak = take(Cmax * 8), o_flag = take((Cmax + 1) * 4), o_grank = take(Cmax * 4),
                 o_ea = take(mmax * 4), o_eb = take(mmax * 4), o_sa = take(mmax * 4),
                 o_sb = take(mmax * 4), o_ss = take(mmax * 8), o_k1 = take(mmax * 8),
                 o_k1b = take(mmax * 8), o_v1 = take(mmax * 4), o_v1b = take(mmax * 4),
                 o_gk = take(Cmax * 8), o_gkb = take(Cmax * 8), o_gv = take(Cmax * 4),
                 o_gvb = take(Cmax * 4), o_start = take((a.B + 1) * 4);
    const size_t o_tmp = take(std::max(radix_sort_scratch_bytes(mmax), radix_sort_scratch_bytes(Cmax)));
    char *base = (char *)ctx_buf(c, S_MERGE, off);
    if (!base) return HOP_ENOMEM;
    uint32_t *cid = (uint32_t *)(base + o_cid);
    uint64_t *ckey = (uint64_t *)(base + o_ckey);
    uint8_t *own = (uint8_t *)(base + o_own);
    uint32_t *parent = (uint32_t *)(base + o_parent), *best = (uint32_t *)(base + o_best),
             *tgt = (uint32_t *)(base + o_tgt), *flag = (uint32_t *)(base + o_flag),
             *grank = (uint32_t *)(base + o_grank), *seg_start = (uint32_t *)(base + o_start);
    unsigned long long *gpeak = (unsigned long long *)(base + o_gpeak);
    uint32_t *ea = (uint32_t *)(base + o_ea), *eb = (uint32_t *)(base + o_eb),
             *sa = (uint32_t *)(base + o_sa), *sb = (uint32_t *)(base + o_sb);
    double *ss = (double *)(base + o_ss);
    uint64_t *k1 = (uint64_t *)(base + o_k1), *k1b = (uint64_t *)(base + o_k1b);
    uint32_t *v1 = (uint32_t *)(base + o_v1), *v1b = (uint32_t *)(base + o_v1b);
    uint64_t *gk = (uint64_t *)(base + o_gk), *gkb = (uint64_t *)(base + o_gkb);
    uint32_t *gv = (uint32_t *)(base + o_gv), *gvb = (uint32_t *)(base + o_gvb);
    void *tmp = base + o_tmp;

    HOP_CUDA(c, cudaMemsetAsync(a.counts, 0, 8 * sizeof(uint32_t), c->stream));
    HOP_CUDA(c, cudaMemsetAsync(a.n_groups, 0, a.B * sizeof(uint32_t), c->stream));
    // M1, M2: dense chain ids of the roots above delta_outer
    root_flag_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(a.chain, a.dkey, n, a.d_o, cid, c->d_err);
    HOP_LAUNCH(c);
    int rc = scan_exclusive_u32(c, cid, cid, n, d_C);
    if (rc) return rc;
    root_list_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(a.chain, a.dkey, n, a.d_o, a.d_p, cid, ckey, own,
                                                            Cmax, c->d_err);
    HOP_LAUNCH(c);
    // M3: strict edge order
    edge_prep_kernel<<<grid_for(c, mmax), 256, 0, c->stream>>>(a.edge_key, a.edge_sum, a.m, n, a.chain, cid,
                                                              a.dkey, a.d_o, ea, eb, k1, v1, c->d_err, Cmax);
    HOP_LAUNCH(c);
    rc = radix_sort_u64_dev(c, k1, k1b, v1, v1b, a.m, 0, 64, tmp);
    if (rc) return rc;
    edge_key2_kernel<<<grid_for(c, mmax), 256, 0, c->stream>>>(a.edge_sum, v1, a.m, k1);
    HOP_LAUNCH(c);
    rc = radix_sort_u64_dev(c, k1, k1b, v1, v1b, a.m, 0, 64, tmp);
    if (rc) return rc;
    edge_permute_kernel<<<grid_for(c, mmax), 256, 0, c->stream>>>(v1, a.m, ea, eb, a.edge_sum, sa, sb, ss);
    HOP_LAUNCH(c);
    // M4, M5: device-bounded rounds
    iota_kernel<<<grid_for(c, Cmax), 256, 0, c->stream>>>(parent, C);
    HOP_LAUNCH(c);
    RoundArgs r{sa, sb, ss, a.m, C, 2.0 * (double)a.d_s, own, parent, best, tgt, d_changed, Cmax, mmax};
    rc = graph_while(c, d_changed, d_round1, kMaxRounds, kErrMergeLoop, proto_round, &r);
    if (rc) return rc;
    rc = graph_while(c, d_changed, d_round2, kMaxRounds, kErrMergeLoop, boruvka_round, &r);
    if (rc) return rc;
    // M6: groups, ranked within their subvolume
    fill_u64_n_kernel<<<grid_for(c, Cmax), 256, 0, c->stream>>>(gpeak, C, 0ull);
    HOP_LAUNCH(c);
    group_peak_kernel<<<grid_for(c, Cmax), 256, 0, c->stream>>>(C, parent, own, ckey, gpeak);
    HOP_LAUNCH(c);
    group_flag_kernel<<<grid_for(c, Cmax), 256, 0, c->stream>>>(C, parent, own, flag);
    HOP_LAUNCH(c);
    uint32_t *gpos = tgt;   // reuse
    rc = scan_exclusive_u32_dev(c, flag, gpos, C, d_G);
    if (rc) return rc;
    group_list_kernel<<<grid_for(c, Cmax), 256, 0, c->stream>>>(C, flag, gpos, gpeak, gk, gv);
    HOP_LAUNCH(c);
    rc = radix_sort_u64_dev(c, gk, gkb, gv, gvb, G, 0, 64, tmp);
    if (rc) return rc;
    group_seg_kernel<<<grid_for(c, Cmax), 256, 0, c->stream>>>(G, gv, ckey, a.seg, a.B, gk, a.n_groups);
    HOP_LAUNCH(c);
    int sub_bits = 0;
    while ((1 << sub_bits) < a.B) sub_bits += 8;
    if (sub_bits) {
        rc = radix_sort_u64_dev(c, gk, gkb, gv, gvb, G, 0, sub_bits, tmp);
        if (rc) return rc;
    }
    rc = scan_exclusive_u32(c, a.n_groups, seg_start, a.B, nullptr);
    if (rc) return rc;
    group_rank_seg_kernel<<<grid_for(c, Cmax), 256, 0, c->stream>>>(G, gv, gk, seg_start, grank);
    HOP_LAUNCH(c);
    particle_group_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(a.chain, a.dkey, n, a.d_o, cid, C, parent,
                                                                own, grank, a.group, c->d_err);
    HOP_LAUNCH(c);
    return HOP_OK;
}
