// HOP steps 2-3 and merging step 3 (Parallel HOP Sec. 2): densest-neighbour
// hops, chains to density peaks, and the chain-pair boundary table.
//
// Keys.  A particle's rank in "density, then smaller index" order is one
// uint64: (density bits << 32) | (0xFFFFFFFF - original index).  Densities
// are >= 0 (or +inf), whose IEEE bits order like the values, so one integer
// compare decides every hop exactly as the oracle's (density, -index) test.
#include "hop_internal.cuh"

#include <algorithm>

namespace {

constexpr uint64_t kEmpty = ~0ull;    // no valid pair key has lo == hi == 0xFFFFFFFF
constexpr int kMaxProbe = 512;
constexpr int kChainLimit = 1 << 26;

__global__ void dkey_kernel(const float *__restrict__ dens, const uint32_t *__restrict__ orig,
                            int64_t n, uint64_t *__restrict__ dkey)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = orig ? orig[i] : (uint32_t)i;
        dkey[i] = ((uint64_t)__float_as_uint(dens[i]) << 32) | (uint64_t)(0xFFFFFFFFu - o);
    }
}

// hop_i = argmax of the key over the first n_hop entries of row i.
__global__ void hop_kernel(const uint64_t *__restrict__ dkey, const uint32_t *__restrict__ nbr,
                           int ld, int64_t n, int n_hop, uint32_t *__restrict__ hop,
                           uint32_t *__restrict__ chain, uint32_t *__restrict__ err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t *row = nbr + i * (int64_t)ld;
        uint32_t best = row[0];
        bool bad = best >= (uint64_t)n;
        uint64_t bk = bad ? 0 : dkey[best];
        for (int t = 1; t < n_hop; ++t) {
            const uint32_t j = row[t];
            if (j >= (uint64_t)n) { bad = true; break; }
            const uint64_t kj = dkey[j];
            if (kj > bk) { bk = kj; best = j; }
        }
        if (bad) {
            atomicOr(err, kErrBadIndex);
            best = (uint32_t)i;
        }
        hop[i] = best;
        chain[i] = best;
    }
}

// Path halving: every pointer moves to its grandparent while walking up.
// Pointers only ever hold ancestors, so walks end at the root; but a thread
// can overwrite another thread's finished root label with an ancestor it
// read earlier, so this pass only shortens paths and chain_root_kernel
// writes the final labels.
__global__ void chain_halving_kernel(uint32_t *chain, int64_t n, uint32_t *err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i;
        int steps = 0;
        for (;;) {
            const uint32_t p = chain[x];
            if (p == x) break;
            const uint32_t gp = chain[p];
            if (gp == p) break;
            chain[x] = gp;
            x = gp;
            if (++steps > kChainLimit) { atomicOr(err, kErrChainLoop); break; }
        }
    }
}

// Final labels: follow pointers (no writes on the way) and store the root.
// Only roots are written, so concurrent walks still end at the root.
__global__ void chain_root_kernel(uint32_t *chain, int64_t n, uint32_t *err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = chain[i];
        int steps = 0;
        for (;;) {
            const uint32_t p = chain[x];
            if (p == x) break;
            x = p;
            if (++steps > kChainLimit) { atomicOr(err, kErrChainLoop); break; }
        }
        chain[i] = x;
    }
}

// A chain label must be a true root of the hop forest.  Rows that do not
// list the particle itself can make hops cycle; following then stops on a
// particle that is not its own hop, which this check reports.
__global__ void chain_check_kernel(const uint32_t *__restrict__ hop, const uint32_t *__restrict__ chain,
                                   int64_t n, uint32_t *__restrict__ err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = chain[i];
        if (hop[r] != r) atomicOr(err, kErrChainLoop);
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdull;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ull;
    z ^= z >> 33;
    return z;
}

__device__ __forceinline__ bool table_insert(uint64_t *hkey, unsigned long long *hval,
                                             uint64_t mask, uint64_t key, unsigned long long v,
                                             unsigned long long *n_ins)
{
    uint64_t h = mix64(key) & mask;
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        uint64_t k = *(volatile uint64_t *)&hkey[h];
        if (k == kEmpty) {
            const unsigned long long prev =
                atomicCAS((unsigned long long *)&hkey[h], (unsigned long long)kEmpty,
                          (unsigned long long)key);
            if (prev == kEmpty) atomicAdd(n_ins, 1ull);
            k = prev == kEmpty ? key : prev;
        }
        if (k == key) {
            if (*(volatile unsigned long long *)&hval[h] < v) atomicMax(&hval[h], v);
            return true;
        }
        h = (h + 1) & mask;
    }
    return false;
}

// Slot of `key`, or -1.  Inserts never probe further than kMaxProbe.
__device__ __forceinline__ int64_t table_find(const uint64_t *hkey, uint64_t mask, uint64_t key)
{
    uint64_t h = mix64(key) & mask;
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        const uint64_t k = hkey[h];
        if (k == key) return (int64_t)h;
        if (k == kEmpty) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// Boundary densities: for i with dens_i >= d_o and j among the first n_merge
// entries of row i (j != i, dens_j >= d_o, chain_i != chain_j), the pair of
// chain labels keeps max(dens_i + dens_j) in fp64 (exact for two fp32).  The
// double is >= 0, so its bits order like its value and atomicMax applies.
// With `directed` the key is (chain_i, chain_j) in that order, so the table
// holds each direction of a pair separately (ADAPTAHOP's symmetric test).
__global__ void boundary_kernel(const uint32_t *__restrict__ chain,
                                const uint64_t *__restrict__ dkey,
                                const uint32_t *__restrict__ nbr, int ld, int64_t n, int n_merge,
                                float d_o, uint64_t *hkey, unsigned long long *hval, uint64_t mask,
                                uint32_t *err, unsigned long long *n_ins, bool directed = false)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float di = key_dens(dkey[i]);
        if (!(di >= d_o)) continue;
        const uint32_t ci = chain[i];
        const uint32_t *row = nbr + i * (int64_t)ld;
        for (int t = 0; t < n_merge; ++t) {
            const uint32_t j = row[t];
            if (j == (uint32_t)i) continue;
            if (j >= (uint64_t)n) { atomicOr(err, kErrBadIndex); continue; }
            const float dj = key_dens(dkey[j]);
            if (!(dj >= d_o)) continue;
            const uint32_t cj = chain[j];
            if (cj == ci) continue;
            const uint64_t key = (directed || ci < cj) ? (((uint64_t)ci << 32) | cj)
                                                       : (((uint64_t)cj << 32) | ci);
            const double s = (double)di + (double)dj;
            if (!table_insert(hkey, hval, mask, key, (unsigned long long)__double_as_longlong(s), n_ins))
                atomicOr(err, kErrTableFull);
        }
    }
}

// Inserts a list of (pair, sum) boundaries into the table; each pair keeps
// its largest sum (the sums are >= 0, so their bits order like the values).
__global__ void edge_insert_kernel(const uint64_t *__restrict__ pair, const double *__restrict__ sum, int64_t m,
                                   uint64_t *hkey, unsigned long long *hval, uint64_t mask, uint32_t *err,
                                   unsigned long long *n_ins)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = pair[e];
        const double s = sum[e];
        if (key == kEmpty || !(s >= 0.0)) {
            atomicOr(err, kErrBadIndex);
            continue;
        }
        if (!table_insert(hkey, hval, mask, key, (unsigned long long)__double_as_longlong(s), n_ins))
            atomicOr(err, kErrTableFull);
    }
}

__global__ void occupied_kernel(const uint64_t *__restrict__ hkey, int64_t cap, uint32_t *__restrict__ occ)
{
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < cap;
         h += (int64_t)gridDim.x * blockDim.x)
        occ[h] = hkey[h] != kEmpty;
}

__global__ void compact_table_kernel(const uint64_t *__restrict__ hkey,
                                     const unsigned long long *__restrict__ hval, int64_t cap,
                                     const uint32_t *__restrict__ pos, uint64_t *__restrict__ ekey,
                                     double *__restrict__ esum)
{
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < cap;
         h += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = hkey[h];
        if (k == kEmpty) continue;
        const uint32_t p = pos[h];
        ekey[p] = k;
        esum[p] = __longlong_as_double((long long)hval[h]);
    }
}

// Symmetric boundaries (ADAPTAHOP, Parallel HOP Sec. 6) from the directed
// table: slot (a, b) with a < b is kept when (b, a) is present too, and
// takes the larger of the two directions' sums.  Only a < b slots are
// written and only a > b slots are read as partners, so there is no race.
__device__ __forceinline__ bool sym_partner(const uint64_t *hkey, uint64_t mask, uint64_t k, int64_t *r)
{
    if (k == kEmpty) return false;
    const uint32_t a = (uint32_t)(k >> 32), b = (uint32_t)k;
    if (a >= b) return false;
    *r = table_find(hkey, mask, ((uint64_t)b << 32) | a);
    return *r >= 0;
}

__global__ void symmetric_flag_kernel(const uint64_t *__restrict__ hkey, unsigned long long *hval, int64_t cap,
                                      uint32_t *__restrict__ flag)
{
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < cap;
         h += (int64_t)gridDim.x * blockDim.x) {
        int64_t r;
        const bool keep = sym_partner(hkey, (uint64_t)cap - 1, hkey[h], &r);
        if (keep && hval[r] > hval[h]) hval[h] = hval[r];
        flag[h] = keep ? 1u : 0u;
    }
}

__global__ void symmetric_compact_kernel(const uint64_t *__restrict__ hkey,
                                         const unsigned long long *__restrict__ hval, int64_t cap,
                                         const uint32_t *__restrict__ pos, uint64_t *__restrict__ ekey,
                                         double *__restrict__ esum)
{
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < cap;
         h += (int64_t)gridDim.x * blockDim.x) {
        int64_t r;
        if (!sym_partner(hkey, (uint64_t)cap - 1, hkey[h], &r)) continue;
        ekey[pos[h]] = hkey[h];
        esum[pos[h]] = __longlong_as_double((long long)hval[h]);
    }
}

__global__ void fill_u64_kernel(uint64_t *p, int64_t n, uint64_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void scatter_kernel(const uint32_t *__restrict__ perm, int64_t n,
                               const float *__restrict__ dens_s, float *__restrict__ dens,
                               const int32_t *__restrict__ group_s, int32_t *__restrict__ group,
                               const uint32_t *__restrict__ nbr_s, int ld_s,
                               uint32_t *__restrict__ nbr, int ld, int n_cols,
                               const uint32_t *__restrict__ chain_s, uint32_t *__restrict__ chain)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = perm[s];
        if (dens) dens[o] = dens_s[s];
        if (group) group[o] = group_s[s];
        if (chain) chain[o] = perm[chain_s[s]];
        if (nbr) {
            const uint32_t *src = nbr_s + s * (int64_t)ld_s;
            uint32_t *dst = nbr + (int64_t)o * ld;
            for (int t = 0; t < n_cols; ++t) dst[t] = perm[src[t]];
        }
    }
}

__global__ void gather_f64_kernel(const double *__restrict__ src, const uint32_t *__restrict__ idx,
                                  int64_t n, double *__restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

}  // namespace

int make_dkey(hop_ctx *c, const float *dens, const uint32_t *orig, int64_t n, uint64_t *dkey)
{
    dkey_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(dens, orig, n, dkey);
    HOP_LAUNCH(c);
    return HOP_OK;
}

int hop_links(hop_ctx *c, const uint64_t *dkey, const uint32_t *nbr, int ld, int64_t n, int n_hop,
              uint32_t *hop, uint32_t *chain)
{
    uint32_t *flag = (uint32_t *)ctx_buf(c, S_MISC, 64);
    if (!flag) return HOP_ENOMEM;
    if (!hop) {
        hop = (uint32_t *)ctx_buf(c, S_HOP, n * sizeof(uint32_t));
        if (!hop) return HOP_ENOMEM;
    }
    HOP_CUDA(c, cudaMemsetAsync(flag, 0, 8, c->stream));
    hop_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(dkey, nbr, ld, n, n_hop, hop, chain, flag);
    HOP_LAUNCH(c);
    chain_halving_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, n, flag);
    HOP_LAUNCH(c);
    chain_root_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, n, flag);
    HOP_LAUNCH(c);
    chain_check_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(hop, chain, n, flag);
    HOP_LAUNCH(c);
    uint32_t *h = (uint32_t *)c->h_pinned;
    HOP_CUDA(c, cudaMemcpyAsync(h, flag, 4, cudaMemcpyDeviceToHost, c->stream));
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h[0] & kErrBadIndex) return ctx_fail(c, HOP_EINVAL, "neighbour index >= n");
    if (h[0] & kErrChainLoop)
        return ctx_fail(c, HOP_ETIMEOUT, "hops contain a cycle (neighbour rows without the particle itself)");
    return HOP_OK;
}

int boundaries_table(hop_ctx *c, const uint32_t *chain, const uint64_t *dkey, const uint32_t *nbr,
                     int ld, int64_t n, int n_merge, float delta_outer, uint64_t **edge_key,
                     double **edge_sum, int64_t *n_edges, bool symmetric)
{
    int64_t cap = 1 << 12;
    while (cap < n / 4 && cap < (int64_t(1) << 31)) cap <<= 1;
    unsigned long long *nins = (unsigned long long *)ctx_buf(c, S_MISC, 64);
    if (!nins) return HOP_ENOMEM;
    unsigned long long *hn = (unsigned long long *)c->h_pinned;
    for (int attempt = 0; attempt < 6; ++attempt) {
        uint64_t *hkey = (uint64_t *)ctx_buf(c, S_HKEY, cap * sizeof(uint64_t));
        unsigned long long *hval = (unsigned long long *)ctx_buf(c, S_HVAL, cap * sizeof(uint64_t));
        if (!hkey || !hval) return HOP_ENOMEM;
        fill_u64_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, cap, kEmpty);
        HOP_LAUNCH(c);
        HOP_CUDA(c, cudaMemsetAsync(hval, 0, cap * sizeof(uint64_t), c->stream));
        HOP_CUDA(c, cudaMemsetAsync(nins, 0, 16, c->stream));
        uint32_t *terr = (uint32_t *)(nins + 1);   // this pass's own error word
        boundary_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, dkey, nbr, ld, n, n_merge,
                                                              delta_outer, hkey, hval,
                                                              (uint64_t)cap - 1, terr, nins, symmetric);
        HOP_LAUNCH(c);
        HOP_CUDA(c, cudaMemcpyAsync(hn, nins, 16, cudaMemcpyDeviceToHost, c->stream));
        HOP_CUDA(c, cudaStreamSynchronize(c->stream));
        const uint32_t e = *(uint32_t *)((char *)hn + 8);
        const int64_t m = (int64_t)hn[0];
        if ((e & kErrBadIndex) != 0) return ctx_fail(c, HOP_EINVAL, "neighbour index >= n");
        if ((e & kErrTableFull) != 0 || m * 10 > cap * 7) {
            cap <<= 2;
            continue;
        }
        uint32_t *occ = (uint32_t *)ctx_buf(c, S_EDGE_TMP, (cap + 1) * sizeof(uint32_t));
        uint64_t *ek = (uint64_t *)ctx_buf(c, S_EDGE_KEY, std::max<int64_t>(m, 1) * sizeof(uint64_t));
        double *es = (double *)ctx_buf(c, S_EDGE_SUM, std::max<int64_t>(m, 1) * sizeof(double));
        if (!occ || !ek || !es) return HOP_ENOMEM;
        if (symmetric) {
            uint32_t *total = terr + 1;
            symmetric_flag_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, hval, cap, occ);
            HOP_LAUNCH(c);
            int rc = scan_exclusive_u32(c, occ, occ, cap, total);
            if (rc) return rc;
            symmetric_compact_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, hval, cap, occ, ek, es);
            HOP_LAUNCH(c);
            HOP_CUDA(c, cudaMemcpyAsync(hn, nins, 16, cudaMemcpyDeviceToHost, c->stream));
            HOP_CUDA(c, cudaStreamSynchronize(c->stream));
            *edge_key = ek;
            *edge_sum = es;
            *n_edges = *(uint32_t *)((char *)hn + 12);
            return HOP_OK;
        }
        occupied_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, cap, occ);
        HOP_LAUNCH(c);
        int rc = scan_exclusive_u32(c, occ, occ, cap, nullptr);
        if (rc) return rc;
        compact_table_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, hval, cap, occ, ek, es);
        HOP_LAUNCH(c);
        *edge_key = ek;
        *edge_sum = es;
        *n_edges = m;
        return HOP_OK;
    }
    return ctx_fail(c, HOP_ENOMEM, "boundary table could not be sized");
}

int edges_max_table(hop_ctx *c, const uint64_t *pair, const double *sum, int64_t m, uint64_t **edge_key,
                    double **edge_sum, int64_t *n_edges)
{
    int64_t cap = 1 << 12;
    while (cap < 2 * m && cap < (int64_t(1) << 31)) cap <<= 1;
    unsigned long long *nins = (unsigned long long *)ctx_buf(c, S_MISC, 64);
    if (!nins) return HOP_ENOMEM;
    unsigned long long *hn = (unsigned long long *)c->h_pinned;
    for (int attempt = 0; attempt < 4; ++attempt) {
        uint64_t *hkey = (uint64_t *)ctx_buf(c, S_HKEY, cap * sizeof(uint64_t));
        unsigned long long *hval = (unsigned long long *)ctx_buf(c, S_HVAL, cap * sizeof(uint64_t));
        if (!hkey || !hval) return HOP_ENOMEM;
        fill_u64_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, cap, kEmpty);
        HOP_LAUNCH(c);
        HOP_CUDA(c, cudaMemsetAsync(hval, 0, cap * sizeof(uint64_t), c->stream));
        HOP_CUDA(c, cudaMemsetAsync(nins, 0, 16, c->stream));
        uint32_t *terr = (uint32_t *)(nins + 1);
        if (m > 0) {
            edge_insert_kernel<<<grid_for(c, m), 256, 0, c->stream>>>(pair, sum, m, hkey, hval, (uint64_t)cap - 1,
                                                                     terr, nins);
            HOP_LAUNCH(c);
        }
        HOP_CUDA(c, cudaMemcpyAsync(hn, nins, 16, cudaMemcpyDeviceToHost, c->stream));
        HOP_CUDA(c, cudaStreamSynchronize(c->stream));
        const uint32_t e = *(uint32_t *)((char *)hn + 8);
        const int64_t u = (int64_t)hn[0];
        if ((e & kErrBadIndex) != 0) return ctx_fail(c, HOP_EINVAL, "a boundary has an empty key or a negative sum");
        if ((e & kErrTableFull) != 0) {
            cap <<= 2;
            continue;
        }
        uint32_t *occ = (uint32_t *)ctx_buf(c, S_EDGE_TMP, (cap + 1) * sizeof(uint32_t));
        uint64_t *ek = (uint64_t *)ctx_buf(c, S_EDGE_KEY, std::max<int64_t>(u, 1) * sizeof(uint64_t));
        double *es = (double *)ctx_buf(c, S_EDGE_SUM, std::max<int64_t>(u, 1) * sizeof(double));
        if (!occ || !ek || !es) return HOP_ENOMEM;
        occupied_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, cap, occ);
        HOP_LAUNCH(c);
        int rc = scan_exclusive_u32(c, occ, occ, cap, nullptr);
        if (rc) return rc;
        compact_table_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, hval, cap, occ, ek, es);
        HOP_LAUNCH(c);
        *edge_key = ek;
        *edge_sum = es;
        *n_edges = u;
        return HOP_OK;
    }
    return ctx_fail(c, HOP_ENOMEM, "boundary table could not be sized");
}

// Graph-safe forms (no host round trip): errors go to the context's error
// word, which the caller reads once the pass has run.
int hop_links_async(hop_ctx *c, const uint64_t *dkey, const uint32_t *nbr, int ld, int64_t n,
                    int n_hop, uint32_t *hop, uint32_t *chain)
{
    hop_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(dkey, nbr, ld, n, n_hop, hop, chain, c->d_err);
    HOP_LAUNCH(c);
    chain_halving_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, n, c->d_err);
    HOP_LAUNCH(c);
    chain_root_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, n, c->d_err);
    HOP_LAUNCH(c);
    chain_check_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(hop, chain, n, c->d_err);
    HOP_LAUNCH(c);
    return HOP_OK;
}

// Boundary table of fixed capacity `cap` (a power of two).  The edge count
// lands in *m_dev; edge_key / edge_sum hold cap entries, the first *m_dev
// valid.  An overfull table sets kErrTableFull in the error word.
int boundaries_table_async(hop_ctx *c, const uint32_t *chain, const uint64_t *dkey,
                           const uint32_t *nbr, int ld, int64_t n, int n_merge, float delta_outer,
                           int64_t cap, uint32_t *m_dev, unsigned long long *nins,
                           uint64_t **edge_key, double **edge_sum)
{
    uint64_t *hkey = (uint64_t *)ctx_buf(c, S_HKEY, cap * sizeof(uint64_t));
    unsigned long long *hval = (unsigned long long *)ctx_buf(c, S_HVAL, cap * sizeof(uint64_t));
    uint32_t *occ = (uint32_t *)ctx_buf(c, S_EDGE_TMP, (cap + 1) * sizeof(uint32_t));
    uint64_t *ek = (uint64_t *)ctx_buf(c, S_EDGE_KEY, cap * sizeof(uint64_t));
    double *es = (double *)ctx_buf(c, S_EDGE_SUM, cap * sizeof(double));
    if (!hkey || !hval || !occ || !ek || !es) return HOP_ENOMEM;
    fill_u64_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, cap, kEmpty);
    HOP_LAUNCH(c);
    HOP_CUDA(c, cudaMemsetAsync(hval, 0, cap * sizeof(uint64_t), c->stream));
    boundary_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(chain, dkey, nbr, ld, n, n_merge, delta_outer,
                                                          hkey, hval, (uint64_t)cap - 1, c->d_err, nins);
    HOP_LAUNCH(c);
    occupied_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, cap, occ);
    HOP_LAUNCH(c);
    int rc = scan_exclusive_u32(c, occ, occ, cap, m_dev);
    if (rc) return rc;
    compact_table_kernel<<<grid_for(c, cap), 256, 0, c->stream>>>(hkey, hval, cap, occ, ek, es);
    HOP_LAUNCH(c);
    *edge_key = ek;
    *edge_sum = es;
    return HOP_OK;
}

int gather_f64(hop_ctx *c, const double *src, const uint32_t *idx, int64_t n, double *dst)
{
    gather_f64_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(src, idx, n, dst);
    HOP_LAUNCH(c);
    return HOP_OK;
}

int scatter_outputs(hop_ctx *c, const uint32_t *perm, int64_t n, const float *dens_s, float *dens,
                    const int32_t *group_s, int32_t *group, const uint32_t *nbr_s, int ld_s,
                    uint32_t *nbr, int ld, int n_cols, const uint32_t *chain_s, uint32_t *chain)
{
    scatter_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(perm, n, dens_s, dens, group_s, group,
                                                         nbr_s, ld_s, nbr, ld, n_cols, chain_s,
                                                         chain);
    HOP_LAUNCH(c);
    return HOP_OK;
}

// ------------------------------------------------------------------------
// hop_link_static: hop_link for callers that cannot allocate device memory.
// Its scratch (density keys, then an error word) lives in this file-scope
// array instead of a context's buffers.  Host code must not pass the
// symbol itself to a kernel: on the host it names a stand-in, not device
// memory.  The device address comes from cudaGetSymbolAddress, looked up
// once per device with that device current.
static __device__ __align__(256) unsigned long long g_link_static_scratch[HOP_STATIC_LINK_MAX_N + 32];

#include <mutex>

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kStaticMaxDevices] = {};
int g_static_sms[kStaticMaxDevices] = {};

// Device address of the scratch array and the SM count of the current device.
int static_scratch(void **ptr, int *sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return HOP_ECUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_link_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HOP_ECUDA;
        }
        int s = 0;
        if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0) {
            cudaGetLastError();
            return HOP_ECUDA;
        }
        g_static_ptr[dev] = p;
        g_static_sms[dev] = s;
    }
    *ptr = g_static_ptr[dev];
    *sms = g_static_sms[dev];
    return HOP_OK;
}

}  // namespace

extern "C" int hop_link_static(const float *dens, const uint32_t *nbr, int32_t ld_nbr, int64_t n,
                               int32_t n_hop, uint32_t *hop, uint32_t *chain, void *cuda_stream)
{
    if (!dens || !nbr || !hop || !chain || n <= 0 || n_hop < 1 || n_hop > ld_nbr) return HOP_EINVAL;
    if (n > HOP_STATIC_LINK_MAX_N) return HOP_ESTATIC;
    void *base = nullptr;
    int sms = 0;
    int rc = static_scratch(&base, &sms);
    if (rc) return rc;
    uint64_t *dkey = (uint64_t *)base;
    uint32_t *flag = (uint32_t *)(dkey + HOP_STATIC_LINK_MAX_N);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int64_t b = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 32);
    const int blocks = (int)std::max<int64_t>(b, 1);
    // the array keeps the previous call's contents: the error word starts at zero
    if (cudaMemsetAsync(flag, 0, 8, st) != cudaSuccess) return HOP_ECUDA;
    dkey_kernel<<<blocks, 256, 0, st>>>(dens, nullptr, n, dkey);
    hop_kernel<<<blocks, 256, 0, st>>>(dkey, nbr, ld_nbr, n, n_hop, hop, chain, flag);
    chain_halving_kernel<<<blocks, 256, 0, st>>>(chain, n, flag);
    chain_root_kernel<<<blocks, 256, 0, st>>>(chain, n, flag);
    chain_check_kernel<<<blocks, 256, 0, st>>>(hop, chain, n, flag);
    if (cudaGetLastError() != cudaSuccess) return HOP_ECUDA;
    uint32_t h = 0;
    if (cudaMemcpyAsync(&h, flag, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HOP_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HOP_ECUDA;
    if (h & kErrBadIndex) return HOP_EINVAL;
    if (h & kErrChainLoop) return HOP_ETIMEOUT;
    return HOP_OK;
}
