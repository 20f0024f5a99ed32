// ADAPTAHOP subhalos on HOP's chains (Parallel HOP Sec. 6, "Parallel HOP
// and Subhalos").
//
//  S1  symmetric boundary table: the directed chain-pair table (both
//      particles >= delta_outer, as in HOP's table), kept only for pairs
//      linked in both directions, each with the larger direction's sum
//      (link.cu, boundaries_table with symmetric = true);
//  S2  dense ids for the chain roots above delta_outer (scan) and, per
//      particle above delta_outer, its root's id;
//  then once per threshold delta_s (the paper's linear cost in the number
//  of thresholds):
//  S3  links with s < 2 delta_s are destroyed; the rest join chains into
//      connected components (hook the larger root under the smaller with
//      atomicMin, compress, repeat until no edge joins two roots);
//  S4  members (dens >= delta_s) give each component its count, fp64
//      density sum and peak key (warp-aggregated atomics);
//  S5  a component is a subhalo when count >= n_min and mean density >=
//      delta_s (1 + f_poisson / sqrt(count)); subhalos are ranked by peak
//      key (radix sort) and every particle gets its rank or -1.
//
// Every per-particle pass reads a few bytes per particle plus one or two
// gathers into the chain arrays, so the levels are HBM- and latency-bound.
#include "hop_internal.cuh"

#include <algorithm>
#include <vector>
#include <cmath>

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kMaxRounds = 64;

// S2: roots above delta_outer; chain labels must be roots of [0, n).
__global__ void sub_root_flag_kernel(const uint32_t *__restrict__ chain, const uint64_t *__restrict__ dkey,
                                 int64_t n, float d_o, uint32_t *__restrict__ flag, uint32_t *__restrict__ err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = chain[i];
        if (c >= (uint64_t)n || chain[c] != c) atomicOr(err, kErrBadIndex);
        flag[i] = (c == (uint32_t)i && key_dens(dkey[i]) >= d_o) ? 1u : 0u;
    }
}

// Per particle above delta_outer: its root's dense id.  A particle above
// delta_outer has a root above it (hops go uphill); anything else is an
// inconsistent input.
__global__ void sub_particle_chain_kernel(const uint32_t *__restrict__ chain, const uint64_t *__restrict__ dkey,
                                      int64_t n, float d_o, const uint32_t *__restrict__ cid,
                                      uint32_t *__restrict__ pc, uint32_t *__restrict__ err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = kNone;
        if (key_dens(dkey[i]) >= d_o) {
            const uint32_t r = chain[i];
            if (r >= (uint64_t)n || !(key_dens(dkey[r]) >= d_o)) atomicOr(err, kErrBadIndex);
            else v = cid[r];
        }
        pc[i] = v;
    }
}

__global__ void sub_edge_ids_kernel(const uint64_t *__restrict__ ekey, int64_t m, int64_t n,
                                const uint32_t *__restrict__ chain, const uint64_t *__restrict__ dkey, float d_o,
                                const uint32_t *__restrict__ cid, uint32_t *__restrict__ ea,
                                uint32_t *__restrict__ eb, uint32_t *__restrict__ err)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t lo = (uint32_t)(ekey[e] >> 32), hi = (uint32_t)ekey[e];
        if (lo >= (uint64_t)n || hi >= (uint64_t)n || chain[lo] != lo || chain[hi] != hi ||
            !(key_dens(dkey[lo]) >= d_o) || !(key_dens(dkey[hi]) >= d_o)) {
            atomicOr(err, kErrBadIndex);
            ea[e] = eb[e] = 0;
            continue;
        }
        ea[e] = cid[lo];
        eb[e] = cid[hi];
    }
}

__global__ void sub_iota_kernel(uint32_t *p, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (uint32_t)i;
}

// S3: one hooking round over the surviving links.
__global__ void sub_hook_kernel(const uint32_t *__restrict__ ea, const uint32_t *__restrict__ eb,
                            const double *__restrict__ es, int64_t m, double two_ds, uint32_t *parent,
                            uint32_t *changed)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!(es[e] >= two_ds)) continue;
        const uint32_t ra = find_root(parent, ea[e]), rb = find_root(parent, eb[e]);
        if (ra == rb) continue;
        atomicMin(&parent[max(ra, rb)], min(ra, rb));
        *changed = 1u;
    }
}

__global__ void sub_compress_kernel(uint32_t *parent, int64_t C)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x)
        parent[c] = find_root(parent, (uint32_t)c);
}

// S4: count, density sum and peak key of every component's members.  The
// sum (fp64 atomics, the slow part) is taken only when the significance
// cut needs it (sum != nullptr).
// The per-particle passes take kSubU elements per thread per batch and
// issue the batch's loads before reducing any of it, so the loads overlap.
// The member pass gives every warp spans of consecutive particles and
// carries its last run of one component on to the next 32 (as the halo
// statistics do), so a large component costs one atomic per span.
constexpr int kSubU = 4;
constexpr int kSubSteps = 32;
constexpr int kSubSpan = 32 * kSubSteps;

__global__ void sub_member_stats_kernel(const uint64_t *__restrict__ dkey, const uint32_t *__restrict__ pc,
                                        int64_t n, float ds, const uint32_t *__restrict__ parent,
                                        unsigned long long *__restrict__ cnt, double *__restrict__ sum,
                                        unsigned long long *__restrict__ pkey)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w0 = w * kSubSpan; w0 < n; w0 += nw * kSubSpan) {
        uint32_t cr = kNone;                  // the carried run: component, count, sum, best key
        unsigned long long cc = 0, cb = 0;
        double csum = 0.0;
        for (int t = 0; t < kSubSteps; t += kSubU) {
            uint64_t k[kSubU];
            uint32_t c[kSubU], r[kSubU];
#pragma unroll
            for (int u = 0; u < kSubU; ++u) {
                const int64_t i = w0 + (int64_t)(t + u) * 32 + lane;
                k[u] = i < n ? dkey[i] : 0ull;
                c[u] = i < n ? pc[i] : kNone;
            }
#pragma unroll
            for (int u = 0; u < kSubU; ++u)
                r[u] = (c[u] != kNone && key_dens(k[u]) >= ds) ? parent[c[u]] : kNone;
#pragma unroll
            for (int u = 0; u < kSubU; ++u) {
                const uint32_t rr = r[u];
                if (!__any_sync(0xffffffffu, rr != kNone)) continue;
                // runs of consecutive lanes in one component
                const uint32_t heads = run_heads((int64_t)rr, lane);
                double sm = sum ? run_sum<double>(heads, lane, rr != kNone ? (double)key_dens(k[u]) : 0.0) : 0.0;
                unsigned long long best = run_max(heads, lane, rr != kNone ? k[u] : 0ull);
                unsigned long long len = (unsigned long long)run_len(heads, lane);
                if (lane == 0 && cr != kNone) {
                    if (rr == cr) {
                        len += cc;
                        sm += csum;
                        best = best > cb ? best : cb;
                    } else {
                        atomicAdd(&cnt[cr], cc);
                        if (sum) atomicAdd(&sum[cr], csum);
                        atomicMax(&pkey[cr], cb);
                    }
                }
                const int last = 31 - __clz(heads);
                if (rr != kNone && ((heads >> lane) & 1u) && lane != last) {
                    atomicAdd(&cnt[rr], len);
                    if (sum) atomicAdd(&sum[rr], sm);
                    atomicMax(&pkey[rr], best);
                }
                cr = __shfl_sync(0xffffffffu, rr, last);
                cc = __shfl_sync(0xffffffffu, len, last);
                csum = __shfl_sync(0xffffffffu, sm, last);
                cb = __shfl_sync(0xffffffffu, best, last);
            }
        }
        if (lane == 0 && cr != kNone) {
            atomicAdd(&cnt[cr], cc);
            if (sum) atomicAdd(&sum[cr], csum);
            atomicMax(&pkey[cr], cb);
        }
    }
}
// S5: the significance cut, in the same fp64 operations as the definition.
// With f = 0 the cut is mean >= delta_s, which every set of members passes:
// each member is >= delta_s, and rounding is monotone, so a running fp64
// sum of N of them is >= N delta_s (exact for a float32 delta_s and
// N < 2^29) and the rounded mean is >= delta_s, in any summation order.
// Then (f = 0 and n < 2^29) sum is nullptr and only the count is tested.
__global__ void sub_accept_kernel(int64_t C, const uint32_t *__restrict__ parent,
                              const unsigned long long *__restrict__ cnt, const double *__restrict__ sum,
                              double ds, long long n_min, double f, uint32_t *__restrict__ flag)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x) {
        uint32_t ok = 0;
        const unsigned long long k = cnt[c];
        if (parent[c] == (uint32_t)c && k > 0 && (long long)k >= n_min) {
            if (!sum) {
                ok = 1u;
            } else {
                const double N = (double)k;
                const double mean = __ddiv_rn(sum[c], N);
                const double thr = __dmul_rn(ds, __dadd_rn(1.0, __ddiv_rn(f, __dsqrt_rn(N))));
                ok = mean >= thr ? 1u : 0u;
            }
        }
        flag[c] = ok;
    }
}

__global__ void sub_list_kernel(int64_t C, const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos,
                            const unsigned long long *__restrict__ pkey, uint64_t *__restrict__ gk,
                            uint32_t *__restrict__ gv)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[c]) continue;
        gk[pos[c]] = ~(uint64_t)pkey[c];   // ascending = peak density desc, index asc
        gv[pos[c]] = (uint32_t)c;
    }
}

__global__ void sub_rank_kernel(DevCount Gc, const uint32_t *__restrict__ gv, uint32_t *__restrict__ rank)
{
    const int64_t G = Gc.get();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x)
        rank[gv[g]] = (uint32_t)g;
}

__global__ void sub_label_kernel(const uint64_t *__restrict__ dkey, const uint32_t *__restrict__ pc, int64_t n,
                                 float ds, const uint32_t *__restrict__ parent, const uint32_t *__restrict__ flag,
                                 const uint32_t *__restrict__ rank, int32_t *__restrict__ sub)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * kSubU;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kSubU; base < n; base += stride) {
        uint64_t k[kSubU];
        uint32_t c[kSubU], r[kSubU];
#pragma unroll
        for (int u = 0; u < kSubU; ++u) {
            const int64_t i = base + (int64_t)u * blockDim.x + threadIdx.x;
            k[u] = i < n ? dkey[i] : 0ull;
            c[u] = i < n ? pc[i] : kNone;
        }
#pragma unroll
        for (int u = 0; u < kSubU; ++u) r[u] = (c[u] != kNone && key_dens(k[u]) >= ds) ? parent[c[u]] : kNone;
#pragma unroll
        for (int u = 0; u < kSubU; ++u) {
            const int64_t i = base + (int64_t)u * blockDim.x + threadIdx.x;
            if (i < n) sub[i] = (r[u] != kNone && flag[r[u]]) ? (int32_t)rank[r[u]] : -1;
        }
    }
}

int subhalos(hop_ctx *c, const uint32_t *chain, const uint64_t *dkey, const uint32_t *nbr, int ld, int64_t n,
             int n_merge, float d_o, const float *levels, int L, int64_t n_min, double f, int32_t *sub,
             int64_t *n_sub)
{
    // S1
    HOP_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
    uint64_t *ek;
    double *es;
    int64_t m;
    int rc = boundaries_table(c, chain, dkey, nbr, ld, n, n_merge, d_o, &ek, &es, &m, true);
    if (rc) return rc;
    HOP_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
    // S2
    uint32_t *hp = (uint32_t *)c->h_pinned;
    // misc: total, then kMaxRounds round flags, then one group count per level
    uint32_t *misc = (uint32_t *)ctx_buf(c, S_MISC, (size_t)(2 + kMaxRounds + L) * sizeof(uint32_t));
    uint32_t *cid = (uint32_t *)ctx_buf(c, S_SUB, (size_t)(2 * n + 64) * sizeof(uint32_t));
    if (!misc || !cid) return HOP_ENOMEM;
    uint32_t *pc = cid + ((n + 1 + 63) & ~int64_t(63));
    uint32_t *d_total = misc, *d_flags = misc + 2, *d_levG = misc + 2 + kMaxRounds;
    HOP_CUDA(c, cudaMemsetAsync(misc, 0, (size_t)(2 + kMaxRounds + L) * sizeof(uint32_t), c->stream));
    sub_root_flag_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, dkey, n, d_o, cid, c->d_err);
    HOP_LAUNCH(c);
    rc = scan_exclusive_u32(c, cid, cid, n, d_total);
    if (rc) return rc;
    sub_particle_chain_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, dkey, n, d_o, cid, pc, c->d_err);
    HOP_LAUNCH(c);
    HOP_CUDA(c, cudaMemcpyAsync(hp, misc, 4, cudaMemcpyDeviceToHost, c->stream));
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    const int64_t C = hp[0];
    // arrays over chains (C) and symmetric boundaries (m)
    const int64_t Cp = std::max<int64_t>(C, 1), mp = std::max<int64_t>(m, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t o_parent = take(Cp * 4), o_cnt = take(Cp * 8), o_sum = take(Cp * 8), o_pkey = take(Cp * 8),
                 o_flag = take((Cp + 1) * 4), o_pos = take((Cp + 1) * 4), o_rank = take(Cp * 4),
                 o_ea = take(mp * 4), o_eb = take(mp * 4), o_gk = take(Cp * 8), o_gkb = take(Cp * 8),
                 o_gv = take(Cp * 4), o_gvb = take(Cp * 4), o_tmp = take(radix_sort_scratch_bytes(Cp));
    char *base = (char *)ctx_buf(c, S_SUB_C, off);
    if (!base) return HOP_ENOMEM;
    uint32_t *parent = (uint32_t *)(base + o_parent), *flag = (uint32_t *)(base + o_flag),
             *gpos = (uint32_t *)(base + o_pos), *rank = (uint32_t *)(base + o_rank),
             *ea = (uint32_t *)(base + o_ea), *eb = (uint32_t *)(base + o_eb);
    unsigned long long *cnt = (unsigned long long *)(base + o_cnt), *pkey = (unsigned long long *)(base + o_pkey);
    double *sum = (double *)(base + o_sum);
    uint64_t *gk0 = (uint64_t *)(base + o_gk), *gkb0 = (uint64_t *)(base + o_gkb);
    uint32_t *gv0 = (uint32_t *)(base + o_gv), *gvb0 = (uint32_t *)(base + o_gvb);
    void *tmp = base + o_tmp;
    if (m > 0) {
        sub_edge_ids_kernel<<<grid_for(c, m), 256, 0, c->stream>>>(ek, m, n, chain, dkey, d_o, cid, ea, eb, c->d_err);
        HOP_LAUNCH(c);
    }
    rc = ctx_check_device_error(c);
    if (rc) return rc;
    c->stats.n_chains = C;
    c->stats.n_edges = m;
    // Each level runs without host round trips except the convergence test
    // of its component rounds, read once per batch of kRoundBatch rounds
    // (rounds after convergence change nothing); group counts stay on the
    // device until every level is enqueued.
    constexpr int kRoundBatch = 4;
    for (int l = 0; l < L; ++l) {
        const float ds = levels[l];
        int32_t *out = sub + (int64_t)l * n;
        if (C == 0) {
            HOP_CUDA(c, cudaMemsetAsync(out, 0xFF, n * sizeof(int32_t), c->stream));
            continue;
        }
        // S3
        sub_iota_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(parent, C);
        HOP_LAUNCH(c);
        int rounds = 0;
        bool converged = m == 0;
        while (!converged) {
            if (rounds + kRoundBatch > kMaxRounds) return ctx_fail(c, HOP_ETIMEOUT, "subhalo components did not converge");
            HOP_CUDA(c, cudaMemsetAsync(d_flags + rounds, 0, kRoundBatch * sizeof(uint32_t), c->stream));
            for (int b = 0; b < kRoundBatch; ++b, ++rounds) {
                sub_hook_kernel<<<grid_for(c, m), 256, 0, c->stream>>>(ea, eb, es, m, 2.0 * (double)ds, parent,
                                                                       d_flags + rounds);
                HOP_LAUNCH(c);
                sub_compress_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(parent, C);
                HOP_LAUNCH(c);
            }
            HOP_CUDA(c, cudaMemcpyAsync(hp + 1, d_flags + rounds - 1, 4, cudaMemcpyDeviceToHost, c->stream));
            HOP_CUDA(c, cudaStreamSynchronize(c->stream));
            converged = hp[1] == 0;
        }
        // S4
        double *lsum = (f > 0.0 || n >= (int64_t(1) << 29)) ? sum : nullptr;
        HOP_CUDA(c, cudaMemsetAsync(cnt, 0, C * 8, c->stream));
        if (lsum) HOP_CUDA(c, cudaMemsetAsync(lsum, 0, C * 8, c->stream));
        HOP_CUDA(c, cudaMemsetAsync(pkey, 0, C * 8, c->stream));
        sub_member_stats_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(dkey, pc, n, ds, parent, cnt, lsum, pkey);
        HOP_LAUNCH(c);
        // S5: accepted components, ranked by peak; their count stays on the device
        sub_accept_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(C, parent, cnt, lsum, (double)ds, (long long)n_min,
                                                                 f, flag);
        HOP_LAUNCH(c);
        rc = scan_exclusive_u32(c, flag, gpos, C, d_levG + l);
        if (rc) return rc;
        const DevCount G{C, d_levG + l};
        sub_list_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(C, flag, gpos, pkey, gk0, gv0);
        HOP_LAUNCH(c);
        uint64_t *gk = gk0, *gkb = gkb0;
        uint32_t *gv = gv0, *gvb = gvb0;
        rc = radix_sort_u64_dev(c, gk, gkb, gv, gvb, G, 0, 64, tmp);
        if (rc) return rc;
        sub_rank_kernel<<<grid_for(c, C), 256, 0, c->stream>>>(G, gv, rank);
        HOP_LAUNCH(c);
        sub_label_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(dkey, pc, n, ds, parent, flag, rank, out);
        HOP_LAUNCH(c);
    }
    std::vector<uint32_t> levG(L);
    HOP_CUDA(c, cudaMemcpyAsync(levG.data(), d_levG, (size_t)L * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                c->stream));
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int l = 0; l < L; ++l) n_sub[l] = C == 0 ? 0 : (int64_t)levG[l];
    return HOP_OK;
}

}  // namespace

extern "C" int hop_subhalos(hop_ctx *c, const uint32_t *chain, const float *dens, const uint32_t *nbr,
                            int32_t ld_nbr, int64_t n, int32_t n_merge, float delta_outer, const float *levels,
                            int32_t n_levels, int64_t n_min, double f_poisson, int32_t *sub, int64_t *n_sub)
{
    if (!c) return HOP_EINVAL;
    c->err.clear();
    if (!chain || !dens || !nbr || !sub || !n_sub || !levels || n <= 0 || n_levels <= 0)
        return ctx_fail(c, HOP_EINVAL, "chain, dens, nbr, levels, sub, n_sub, n > 0 and n_levels > 0 are required");
    if (n >= (int64_t(1) << 31) - 1) return ctx_fail(c, HOP_EINVAL, "n must be < 2^31 - 1");
    if (n_merge < 1 || n_merge > ld_nbr) return ctx_fail(c, HOP_EINVAL, "n_merge must be in [1, ld_nbr]");
    if (n_min < 1) return ctx_fail(c, HOP_EINVAL, "n_min must be >= 1");
    if (!(f_poisson >= 0.0) || !std::isfinite(f_poisson)) return ctx_fail(c, HOP_EINVAL, "f_poisson must be >= 0");
    for (int l = 0; l < n_levels; ++l)
        if (!std::isfinite(levels[l]) || !(levels[l] >= delta_outer))
            return ctx_fail(c, HOP_EINVAL, "every level must be finite and >= delta_outer");
    HOP_CUDA(c, cudaSetDevice(c->device));
    const int64_t launches0 = c->launches;
    HOP_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    uint64_t *dkey = (uint64_t *)ctx_buf(c, S_DKEY, n * sizeof(uint64_t));
    if (!dkey) return HOP_ENOMEM;
    int rc = make_dkey(c, dens, nullptr, n, dkey);
    if (rc) return rc;
    rc = subhalos(c, chain, dkey, nbr, ld_nbr, n, n_merge, delta_outer, levels, n_levels, n_min, f_poisson, sub,
                  n_sub);
    if (rc) return rc;
    HOP_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    const int e = ctx_check_device_error(c);
    float ms = 0.f, ms_b = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]) != cudaSuccess) cudaGetLastError();
    if (cudaEventElapsedTime(&ms_b, c->ev[2], c->ev[3]) != cudaSuccess) cudaGetLastError();
    c->stats.ms_total = ms;
    c->stats.ms_boundaries = ms_b;
    c->stats.ms_merge = ms - ms_b;
    c->stats.launches = c->launches - launches0;
    return e;
}
