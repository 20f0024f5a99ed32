// Device-wide exclusive scan and a stable LSD radix sort of (uint64 key,
// uint32 value) pairs, 8 bits per pass.  Used to order particles by Morton
// key (the cell-grid build), and for small sorts in the merge.
#include "hop_internal.cuh"

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096
constexpr int kSortWarps = kSortThreads / 32;

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Block-wide exclusive scan of one value per thread; returns the thread's
// exclusive prefix and writes the block total to *total.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *smem_warp, uint32_t *total)
{
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < (uint32_t)nw ? smem_warp[lane] : 0u;
        uint32_t s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= (uint32_t)o) s += y;
        }
        if (lane < (uint32_t)nw) smem_warp[lane] = s - w;
        if (lane == (uint32_t)nw - 1) smem_warp[32] = s;
    }
    __syncthreads();
    uint32_t r = smem_warp[warp] + x - v;
    *total = smem_warp[32];
    __syncthreads();
    return r;
}

__global__ void scan_reduce_kernel(const uint32_t *__restrict__ in, DevCount nc,
                                   uint32_t *__restrict__ partial)
{
    __shared__ uint32_t sw[33];
    const int64_t n = nc.get();
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    uint32_t tot;
    block_exclusive_scan(s, sw, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Each thread owns kScanItems consecutive items.
__global__ void scan_apply_kernel(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                  DevCount nc, const uint32_t *__restrict__ partial_scanned,
                                  uint32_t *__restrict__ total_dev, int write_total)
{
    __shared__ uint32_t sw[33];
    const int64_t n = nc.get();
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        int64_t i = base + r;
        v[r] = i < n ? in[i] : 0u;
        s += v[r];
    }
    uint32_t tot;
    uint32_t pre = block_exclusive_scan(s, sw, &tot);
    pre += partial_scanned ? partial_scanned[blockIdx.x] : 0u;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        int64_t i = base + r;
        if (i < n) out[i] = pre;
        pre += v[r];
    }
    if (write_total && total_dev && threadIdx.x == blockDim.x - 1 && blockIdx.x == gridDim.x - 1)
        *total_dev = pre;
}

// ------------------------------------------------------------ radix sort --

__global__ void radix_hist_kernel(const uint64_t *__restrict__ keys, DevCount nc, int shift,
                                  int64_t nblocks, uint32_t *__restrict__ counts)
{
    __shared__ uint32_t hist[256];
    const int64_t n = nc.get();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        uint32_t d = valid ? (uint32_t)((keys[i] >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t leader = __ffs(peers) - 1;
        if (valid && lane_id() == leader) atomicAdd(&hist[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x)
        counts[(int64_t)d * nblocks + blockIdx.x] = hist[d];
}

// Stable scatter through a tile-local sort.  A block takes 4096 items: warp
// w ranks its 512 (16 rounds of 32 consecutive items, input order) per digit
// with match/popc and its own digit counters; a scan over (digit, warp)
// gives each item its position in the tile sorted by digit; the tile is
// rebuilt in shared memory in that order and written out in order, so each
// digit's run goes to consecutive global addresses.
constexpr int kLsSmem = kSortWarps * 256 * 4 + 256 * 4 * 2 + kSortTile * 12;

__global__ void __launch_bounds__(kSortThreads, 2) radix_local_scatter_kernel(
    const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint64_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, DevCount nc, int shift, int64_t nblocks, const uint32_t *__restrict__ offsets)
{
    extern __shared__ __align__(16) unsigned char ls_raw[];
    uint32_t *wcnt = (uint32_t *)ls_raw;                       // [warp][digit]
    uint32_t *lstart = wcnt + kSortWarps * 256;                // digit -> first tile position
    uint32_t *gbase = lstart + 256;                            // digit -> global position of tile position 0
    uint64_t *skey = (uint64_t *)(gbase + 256);
    uint32_t *sval = (uint32_t *)(skey + kSortTile);
    const int64_t n = nc.get();
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t lt = lanemask_lt();
    const int64_t tile = (int64_t)blockIdx.x * kSortTile;
    for (int t = threadIdx.x; t < kSortWarps * 256; t += kSortThreads) wcnt[t] = 0;
    __syncthreads();
    uint64_t key[kSortItems];
    uint32_t val[kSortItems], rnk[kSortItems];
    uint32_t *mycnt = wcnt + warp * 256;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = tile + (int64_t)warp * (32 * kSortItems) + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? keys_in[i] : 0ull;
        val[r] = valid ? vals_in[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = tile + (int64_t)warp * (32 * kSortItems) + r * 32 + lane;
        const bool valid = i < n;
        const uint32_t d = valid ? (uint32_t)((key[r] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t leader = __ffs(peers) - 1;
        uint32_t prior = 0;
        if (valid && lane == leader) {
            prior = mycnt[d];
            mycnt[d] = prior + __popc(peers);
        }
        prior = __shfl_sync(0xffffffffu, prior, leader);
        rnk[r] = prior + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    {
        // digit d = threadIdx.x: the runs of the 8 warps, then the tile scan
        const uint32_t d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w * 256 + d];
            wcnt[w * 256 + d] = run;
            run += c;
        }
        __shared__ uint32_t sw[33];
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(run, sw, &tot);
        lstart[d] = ex;
        gbase[d] = offsets[(int64_t)d * nblocks + blockIdx.x] - ex;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) wcnt[w * 256 + d] += ex;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = tile + (int64_t)warp * (32 * kSortItems) + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)((key[r] >> shift) & 255u);
            const uint32_t p = mycnt[d] + rnk[r];
            skey[p] = key[r];
            sval[p] = val[r];
        }
    }
    __syncthreads();
    const int64_t m = n - tile < kSortTile ? n - tile : kSortTile;
    for (int p = threadIdx.x; p < m; p += kSortThreads) {
        const uint64_t k = skey[p];
        const uint32_t d = (uint32_t)((k >> shift) & 255u);
        const uint32_t dst = gbase[d] + (uint32_t)p;
        keys_out[dst] = k;
        vals_out[dst] = sval[p];
    }
}

__global__ void iota_kernel(uint32_t *out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)i;
}

}  // namespace

// Scratch for the scan: partial sums for every recursion level.
static size_t scan_scratch_elems(int64_t n)
{
    size_t tot = 0;
    int64_t m = n;
    while (m > kScanTile) {
        m = (m + kScanTile - 1) / kScanTile;
        tot += (size_t)m + 64;
    }
    return tot + 64;
}

static int scan_rec(hop_ctx *c, const uint32_t *in, uint32_t *out, DevCount n, uint32_t *scratch,
                    uint32_t *total_dev)
{
    const int64_t nb = (n.max + kScanTile - 1) / kScanTile;
    if (nb <= 1) {
        scan_apply_kernel<<<1, kScanThreads, 0, c->stream>>>(in, out, n, nullptr, total_dev, 1);
        HOP_LAUNCH(c);
        return HOP_OK;
    }
    uint32_t *partial = scratch;
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, partial);
    HOP_LAUNCH(c);
    int rc = scan_rec(c, partial, partial, DevCount{nb, nullptr}, scratch + nb + 64, total_dev);
    if (rc) return rc;
    scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, out, n, partial, nullptr, 0);
    HOP_LAUNCH(c);
    return HOP_OK;
}

int scan_exclusive_u32(hop_ctx *c, const uint32_t *in, uint32_t *out, int64_t n,
                       uint32_t *total_dev)
{
    return scan_exclusive_u32_dev(c, in, out, DevCount{n, nullptr}, total_dev);
}

// Items [0, n.get()) are scanned; the grid covers n.max.
int scan_exclusive_u32_dev(hop_ctx *c, const uint32_t *in, uint32_t *out, DevCount n,
                           uint32_t *total_dev)
{
    if (n.max <= 0) {
        if (total_dev) HOP_CUDA(c, cudaMemsetAsync(total_dev, 0, 4, c->stream));
        return HOP_OK;
    }
    uint32_t *scratch = (uint32_t *)ctx_buf(c, S_SCAN, scan_scratch_elems(n.max) * sizeof(uint32_t));
    if (!scratch) return HOP_ENOMEM;
    return scan_rec(c, in, out, n, scratch, total_dev);
}

size_t radix_sort_scratch_bytes(int64_t n)
{
    int64_t nb = (n + kSortTile - 1) / kSortTile;
    return (size_t)(256 * nb + 64) * sizeof(uint32_t);
}

// Sorts (keys, vals) by key bits [begin_bit, end_bit).  On return `keys` and
// `vals` point at the sorted arrays (the pointers are swapped with the
// *_alt buffers as passes ping-pong).
int radix_sort_u64(hop_ctx *c, uint64_t *&keys, uint64_t *&keys_alt, uint32_t *&vals,
                   uint32_t *&vals_alt, int64_t n, int begin_bit, int end_bit, void *scratch)
{
    if (n <= 1) return HOP_OK;
    return radix_sort_u64_dev(c, keys, keys_alt, vals, vals_alt, DevCount{n, nullptr}, begin_bit,
                              end_bit, scratch);
}

// Sorts the first n.get() pairs; the grid and the scratch cover n.max.  The
// number of passes is fixed by the bit range, so the result lands in the
// same buffer whatever the device count.
int radix_sort_u64_dev(hop_ctx *c, uint64_t *&keys, uint64_t *&keys_alt, uint32_t *&vals,
                       uint32_t *&vals_alt, DevCount n, int begin_bit, int end_bit, void *scratch)
{
    if (n.max <= 0) return HOP_OK;
    const int64_t nb = (n.max + kSortTile - 1) / kSortTile;
    uint32_t *counts = (uint32_t *)scratch;
    HOP_CUDA(c, cudaFuncSetAttribute(radix_local_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kLsSmem));
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        radix_hist_kernel<<<(unsigned)nb, kSortThreads, 0, c->stream>>>(keys, n, shift, nb, counts);
        HOP_LAUNCH(c);
        int rc = scan_exclusive_u32(c, counts, counts, 256 * nb, nullptr);
        if (rc) return rc;
        radix_local_scatter_kernel<<<(unsigned)nb, kSortThreads, kLsSmem, c->stream>>>(
            keys, vals, keys_alt, vals_alt, n, shift, nb, counts);
        HOP_LAUNCH(c);
        uint64_t *tk = keys; keys = keys_alt; keys_alt = tk;
        uint32_t *tv = vals; vals = vals_alt; vals_alt = tv;
    }
    return HOP_OK;
}

int iota_u32(hop_ctx *c, uint32_t *out, int64_t n)
{
    if (n <= 0) return HOP_OK;
    int blocks = (int)((n + 255) / 256);
    if (blocks > c->num_sms * 16) blocks = c->num_sms * 16;
    iota_kernel<<<blocks, 256, 0, c->stream>>>(out, n);
    HOP_LAUNCH(c);
    return HOP_OK;
}
