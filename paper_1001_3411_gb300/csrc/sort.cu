// Device-wide exclusive scan and a stable LSD radix sort of (uint64 key,
// uint32 value) pairs, 8 bits per pass.  Used to order particles by Morton
// key (the cell-grid build), and for small sorts in the merge.
#include "hop_internal.cuh"

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096

constexpr int kSortThreads = 256;
constexpr int kSortItems = 12;
constexpr int kSortTile = kSortThreads * kSortItems;   // 3072
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
//
// Stable LSD radix sort, 8 bits per pass, one read and one write of the
// (key, value) pairs per pass.  One kernel counts the digits of every pass
// up front; a pass then needs, for each tile of 3072 items and each digit,
// how many items of that digit the earlier tiles hold.  Tiles are taken in
// input order from a counter, so every earlier tile is already running: a
// tile publishes its own digit counts, then walks back over its
// predecessors' published words, adding counts until it meets a prefix
// that is already complete, and publishes its own complete prefix
// (decoupled look-back, Merrill & Garland 2016).

constexpr uint64_t kStLocal = 1ull << 62;       // word holds this tile's count only
constexpr uint64_t kStIncl = 2ull << 62;        // word holds the count of every tile up to this one
constexpr uint64_t kStValue = (1ull << 62) - 1;
constexpr int kLookbackSpins = 1 << 22;         // limit of a look-back wait (kErrSortWait)
constexpr int kLookbackWindow = 4;              // predecessors read at once
constexpr int kMaxPasses = 8;

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Digit counts of passes [0, npass) (pass p: bits shift0 + 8p ..) over the
// first nc.get() keys, summed into counts[p * 256 + d] (zeroed by the caller).
// Each warp adds into one of kDigitCopies shared copies, which spreads the
// same-address atomics of clustered keys.
constexpr int kDigitCopies = 4;

__global__ void radix_digits_kernel(const uint64_t *__restrict__ keys, DevCount nc, int shift0, int npass,
                                    uint32_t *__restrict__ counts)
{
    __shared__ uint32_t hist[kDigitCopies * kMaxPasses * 256];
    const int64_t n = nc.get();
    const int span = npass * 256;
    for (int t = threadIdx.x; t < kDigitCopies * span; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    uint32_t *h = hist + ((threadIdx.x >> 5) % kDigitCopies) * span;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = keys[i];
        for (int p = 0; p < npass; ++p) atomicAdd(&h[p * 256 + (uint32_t)((k >> (shift0 + 8 * p)) & 255u)], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        uint32_t v = 0;
#pragma unroll
        for (int c = 0; c < kDigitCopies; ++c) v += hist[c * span + t];
        if (v) atomicAdd(&counts[t], v);
    }
}

// One pass.  A block takes the next tile from *tile_ctr; warp w ranks its
// 384 items (12 rounds of 32 consecutive items, input order) per digit with
// ballots/popc and its own digit counters; a scan over (digit, warp) gives
// each item its position in the tile sorted by digit; the look-back gives
// each digit's global position; the tile is rebuilt in shared memory in
// digit order and written out in order, so each digit's run goes to
// consecutive global addresses.  `status` (one word per tile and digit) and
// *tile_ctr are zero on entry.
constexpr int kLsSmem = kSortWarps * 256 * 4 + 256 * 4 + kSortTile * 12;

__global__ void __launch_bounds__(kSortThreads, 3) radix_onesweep_kernel(
    const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint64_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, DevCount nc, int shift, const uint32_t *__restrict__ digit_count,
    uint64_t *__restrict__ status, uint32_t *__restrict__ tile_ctr, uint32_t *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char ls_raw[];
    uint32_t *wcnt = (uint32_t *)ls_raw;                       // [warp][digit]
    uint32_t *gbase = wcnt + kSortWarps * 256;                 // digit -> global position of tile position 0
    uint64_t *skey = (uint64_t *)(gbase + 256);
    uint32_t *sval = (uint32_t *)(skey + kSortTile);
    __shared__ uint32_t sw[33];
    __shared__ uint32_t s_tile, s_bad;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(tile_ctr, 1u);
        s_bad = 0;
    }
    for (int t = threadIdx.x; t < kSortWarps * 256; t += kSortThreads) wcnt[t] = 0;
    __syncthreads();
    const int64_t n = nc.get();
    const uint32_t t_id = s_tile;
    const int64_t tile = (int64_t)t_id * kSortTile;
    if (tile >= n) return;                                     // whole block: no item, no later tile has any
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t lt = lanemask_lt();
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
        // lanes with the same digit: eight ballots, one per digit bit (a
        // warp match costs more here)
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
        if (!valid) peers = ~peers;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint32_t vb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? vb : ~vb;
        }
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
        // digit d = threadIdx.x: the runs of the 8 warps, the tile scan, the
        // look-back over earlier tiles
        const uint32_t d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w * 256 + d];
            wcnt[w * 256 + d] = run;
            run += c;
        }
        uint64_t *mine = status + (int64_t)t_id * 256 + d;
        st_relaxed_u64(mine, (t_id == 0 ? kStIncl : kStLocal) | run);
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(run, sw, &tot);
        const uint32_t gstart = block_exclusive_scan(digit_count[d], sw, &tot);
        uint64_t before = 0;
        if (t_id > 0) {
            // predecessors are read kLookbackWindow at a time (independent
            // loads), then consumed in order up to the first complete prefix
            int64_t j = (int64_t)t_id - 1;
            int spins = 0;
            for (;;) {
                uint64_t x[kLookbackWindow];
#pragma unroll
                for (int u = 0; u < kLookbackWindow; ++u)
                    x[u] = j - u >= 0 ? ld_relaxed_u64(status + (j - u) * 256 + d) : 0ull;
                int used = 0;
                bool done = false, stalled = false;
#pragma unroll
                for (int u = 0; u < kLookbackWindow; ++u) {
                    if (done || stalled) continue;
                    if ((x[u] >> 62) == 0) {
                        stalled = true;                        // not published yet: read again from here
                        continue;
                    }
                    before += x[u] & kStValue;
                    ++used;
                    done = (x[u] & kStIncl) != 0;              // tile 0's word is complete, so j stays >= 0
                }
                if (done) break;
                j -= used;
                if (used == 0 && (++spins & 255) == 0 &&
                    (spins >= kLookbackSpins || (ld_relaxed_u32(err) & kErrSortWait))) {
                    atomicOr(err, kErrSortWait);
                    s_bad = 1;
                    break;
                }
            }
            st_relaxed_u64(mine, kStIncl | (before + run));
        }
        gbase[d] = gstart + (uint32_t)before - ex;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) wcnt[w * 256 + d] += ex;
    }
    __syncthreads();
    if (s_bad) return;
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
        if (dst < (uint64_t)n) {
            keys_out[dst] = k;
            vals_out[dst] = sval[p];
        }
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

// Scratch: the digit counts of every pass, the tile counter, then one
// look-back word per tile and digit.
static int64_t sort_tiles(int64_t n) { return (n + kSortTile - 1) / kSortTile; }
constexpr size_t kSortHead = kMaxPasses * 256 * 4 + 256;

size_t radix_sort_scratch_bytes(int64_t n)
{
    return kSortHead + (size_t)sort_tiles(n < 1 ? 1 : n) * 256 * sizeof(uint64_t);
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
    if (n.max <= 0 || end_bit <= begin_bit) return HOP_OK;
    const int npass = (end_bit - begin_bit + 7) / 8;
    if (npass > kMaxPasses) return ctx_fail(c, HOP_EINVAL, "radix sort over more than 64 key bits");
    const int64_t nb = sort_tiles(n.max);
    uint32_t *counts = (uint32_t *)scratch;
    uint32_t *tile_ctr = (uint32_t *)((char *)scratch + kMaxPasses * 256 * 4);
    uint64_t *status = (uint64_t *)((char *)scratch + kSortHead);
    HOP_CUDA(c, cudaFuncSetAttribute(radix_onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kLsSmem));
    HOP_CUDA(c, cudaMemsetAsync(counts, 0, (size_t)npass * 256 * 4, c->stream));
    const int hb = (int)std::min<int64_t>((n.max + 255) / 256, (int64_t)c->num_sms * 4);
    radix_digits_kernel<<<hb, 256, 0, c->stream>>>(keys, n, begin_bit, npass, counts);
    HOP_LAUNCH(c);
    for (int p = 0; p < npass; ++p) {
        HOP_CUDA(c, cudaMemsetAsync(tile_ctr, 0, 256 + (size_t)nb * 256 * sizeof(uint64_t), c->stream));
        radix_onesweep_kernel<<<(unsigned)nb, kSortThreads, kLsSmem, c->stream>>>(
            keys, vals, keys_alt, vals_alt, n, begin_bit + 8 * p, counts + p * 256, status, tile_ctr, c->d_err);
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
