// Certified cell-stencil kNN fused with the M4 cubic-spline density (HOP
// step 1, Parallel HOP Sec. 2): the count-then-gather kernel for float32
// positions, P lanes per query (Q = 32 / P queries per warp).
//
// Work unit.  A warp takes a chunk of Q consecutive Morton-sorted particles
// (one subvolume).  Consecutive queries farther apart than the chunk's first
// radius start a new group; each group is searched on its own, so a chunk
// that straddles a jump of the Morton curve scans compact regions.  A
// group's region is its queries' bounding box grown by the search radius:
// the warp walks the cells (side >= radius / cpr) that meet it, stages their
// particles in shared memory (a staged particle must itself lie within the
// radius of the box) and the P lanes of every query split the staged
// particles between them.
//
// Scan A (count).  Each lane counts, in its own shared-memory histogram row,
// the staged particles within R of its query, in 64 quarter-octave bins of
// d^2 below R^2 (the lowest bin is open).  A query whose rows hold fewer
// than Ndens particles is not certified: the group repeats with a larger R.
// Otherwise the rows give the bin holding the Ndens-th nearest and the bin
// holding the Nhop-th nearest.  When the Ndens-th bin is crowded (a dense
// clump at that distance) the same scan counts again in 64 finer bins of
// that bin, until the list below fits.
//
// Scan B (gather).  The group scans again with the (smaller) radius that
// covers every query's Ndens-th bin and keeps, per query, exactly the
// particles up to that bin: about Ndens plus the bin's own entries.
//
// Selection.  The exact Ndens-th d^2 is ranked among the entries of its bin;
// the density is a fixed-point sum of w(2 r / r_k) over the list (so it does
// not depend on the order the entries arrive in); the Nhop nearest are
// ranked by (d^2, original index) among the entries up to their bin.
//
// Results equal those of the other kNN kernels bit for bit: the same
// per-component minimum-image differences (a coordinate >= L/2 moves by -L
// exactly where the region crosses a face), the same fused d^2, the same
// exact k-th distance, list order and fixed-point density sum.
#include "hop_internal.cuh"
#include "knn_common.cuh"

#include <math.h>

namespace {

constexpr uint32_t kAll = 0xffffffffu;
constexpr int kCgWarps = 4;                 // warps per block
constexpr int kCgTile = 128;                // staged candidates per tile
constexpr int kCgPer = kCgTile / 32;        // candidates each lane fetches per tile
constexpr int kBins = 64;                   // histogram bins per lane row
constexpr int kShift0 = 21;                 // first window: quarter octaves of d^2
constexpr int kKC = 32;                     // entries of the k-th bin ranked in a small list
constexpr int kOC = 32;                     // candidates for the n_out nearest ranked in a small list
constexpr int kCgTries = 96;
constexpr int kRefine = 12;                 // window refinements of a crowded k-th bin

struct Cand {
    float x, y, z;
    uint32_t s;
};

struct CgDev {
    const float4 *spos;
    const uint64_t *keys;
    const uint32_t *cellT;
    int level_dense;
    int64_t n, n_chunks;
    float box, inv_box, half_box, norm;
    int k, n_out, ld_out, capq;
    const float *chunk_r;
    float plain_r;
    int cpr;
    const SegDesc *seg;
    int B;
    uint32_t *nbr_s;
    float *dens_s;
    float *rk_s;
    unsigned long long *chunk_counter, *counters;
    uint32_t *err;
};

// Shared memory of one warp, byte offsets.  The histogram rows (scan A) and
// the per-query lists with their small selection arrays (scan B and the
// selection) share one region.
template <int Q> struct CgSmem {
    static constexpr size_t tile = 0;                                        // kCgTile + 32 candidates
    static constexpr size_t rs = tile + sizeof(Cand) * (kCgTile + 32);       // 32 range starts
    static constexpr size_t ro = rs + 32 * 4;                                // 33 prefix offsets
    static constexpr size_t uni = (ro + 33 * 4 + 15) & ~size_t(15);
    static constexpr size_t hist_bytes = (size_t)kBins * 32 * 4;
    __host__ __device__ static size_t ld(int) { return uni; }
    __host__ __device__ static size_t ls(int capq) { return uni + (size_t)Q * capq * 4; }
    __host__ __device__ static size_t kd(int capq) { return uni + (size_t)Q * capq * 8; }
    __host__ __device__ static size_t od(int capq) { return kd(capq) + (size_t)Q * kKC * 4; }
    __host__ __device__ static size_t os(int capq) { return od(capq) + (size_t)Q * kOC * 4; }
    __host__ __device__ static size_t total(int capq)
    {
        const size_t lists = os(capq) + (size_t)Q * kOC * 4 - uni;
        const size_t u = lists > hist_bytes ? lists : hist_bytes;
        return (uni + u + 15) & ~size_t(15);
    }
};

__device__ __forceinline__ float cg_wmin(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kAll, v, o));
    return v;
}
__device__ __forceinline__ float cg_wmax(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kAll, v, o));
    return v;
}
__device__ __forceinline__ int cg_wmax_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kAll, v, o));
    return v;
}
// Sum over the P lanes of a query group (all 32 lanes call it).
template <int P> __device__ __forceinline__ int gsum(int v)
{
#pragma unroll
    for (int o = 1; o < P; o <<= 1) v += __shfl_xor_sync(kAll, v, o);
    return v;
}
template <int P> __device__ __forceinline__ float gmaxf(float v)
{
#pragma unroll
    for (int o = 1; o < P; o <<= 1) v = fmaxf(v, __shfl_xor_sync(kAll, v, o));
    return v;
}

// Distance from [a, b] to [lo, hi] along one axis, made smaller by eps so
// that rounding never drops a needed cell or particle.
__device__ __forceinline__ float cg_gap(float a, float b, float lo, float hi, float eps)
{
    return fmaxf(0.f, fmaxf(lo - b, a - hi) - eps);
}

// Largest float (as bits) in window bin i: bins are bits >> shift relative
// to base = top - (kBins - 1); bin 0 is open below.
__device__ __forceinline__ float bin_edge(int base, int shift, int i)
{
    const long long e = ((long long)(base + i + 1) << shift) - 1;
    if (e < 0) return -1.f;
    if (e >= 0x7f800000ll) return __uint_as_float(0x7f7fffffu);
    return __uint_as_float((uint32_t)e);
}

// The region of a query group for radius r: frame flags and the members'
// bounding box in frame coordinates, and the cells to visit.
struct Region {
    bool full, pw, wx, wy, wz;
    float flx, fhx, fly, fhy, flz, fhz;
    float r, r2c;
    int l, G;
    float csz;
    int c0x, c0y, c0z, nx, ny, nz;
};

__device__ __forceinline__ Region make_region(bool member, float rqx, float rqy, float rqz, float r, float box,
                                              float half, float inv_box, int cpr)
{
    Region g;
    g.full = 2.f * r >= half;
    g.r = r;
    g.r2c = r * r * 1.00001f + box * box * 1e-12f;
    const float lx = cg_wmin(member ? rqx : INFINITY), hx = cg_wmax(member ? rqx : -INFINITY);
    const float ly = cg_wmin(member ? rqy : INFINITY), hy = cg_wmax(member ? rqy : -INFINITY);
    const float lz = cg_wmin(member ? rqz : INFINITY), hz = cg_wmax(member ? rqz : -INFINITY);
    g.wx = lx - r < 0.f || hx + r >= box;
    g.wy = ly - r < 0.f || hy + r >= box;
    g.wz = lz - r < 0.f || hz + r >= box;
    // a region crossing a face and also L/2 on that axis cannot use one
    // frame: then each pair takes its own minimum image
    const bool mixed = (g.wx && lx - r < half && half <= hx + r) || (g.wy && ly - r < half && half <= hy + r) ||
                       (g.wz && lz - r < half && half <= hz + r);
    g.pw = g.full || mixed;
    const float qx = (!g.pw && g.wx && rqx >= half) ? rqx - box : rqx;
    const float qy = (!g.pw && g.wy && rqy >= half) ? rqy - box : rqy;
    const float qz = (!g.pw && g.wz && rqz >= half) ? rqz - box : rqz;
    g.flx = cg_wmin(member ? qx : INFINITY);
    g.fhx = cg_wmax(member ? qx : -INFINITY);
    g.fly = cg_wmin(member ? qy : INFINITY);
    g.fhy = cg_wmax(member ? qy : -INFINITY);
    g.flz = cg_wmin(member ? qz : INFINITY);
    g.fhz = cg_wmax(member ? qz : -INFINITY);
    g.l = 1;
    g.G = 2;
    g.c0x = g.c0y = g.c0z = 0;
    g.nx = g.ny = g.nz = 1;
    if (!g.full) {
        const float cells = box * (float)cpr / r;   // 2^l <= cells: side >= r / cpr
        while (g.l < kMaxLevel && (float)(1 << (g.l + 1)) <= cells) ++g.l;
        g.G = 1 << g.l;
        const float sc = inv_box * (float)g.G;
        g.c0x = (int)floorf((g.flx - r) * sc);
        g.c0y = (int)floorf((g.fly - r) * sc);
        g.c0z = (int)floorf((g.flz - r) * sc);
        g.nx = (int)floorf((g.fhx + r) * sc) - g.c0x + 1;
        g.ny = (int)floorf((g.fhy + r) * sc) - g.c0y + 1;
        g.nz = (int)floorf((g.fhz + r) * sc) - g.c0z + 1;
        if (g.nx >= g.G) { g.c0x = 0; g.nx = g.G; }
        if (g.ny >= g.G) { g.c0y = 0; g.ny = g.G; }
        if (g.nz >= g.G) { g.c0z = 0; g.nz = g.G; }
    }
    g.csz = box / (float)g.G;
    return g;
}

// Walks the cells of region g, stages their particles (those within g.r of
// the members' box) in tiles of up to kCgTile and calls fn(m) on each tile of
// m staged candidates (padded with NaN entries to a multiple of 32).  All
// lanes call it; the tile is valid until fn returns.
template <typename F>
__device__ __forceinline__ void scan_region(const Region &g, const float4 *__restrict__ spos,
                                            const uint64_t *__restrict__ keys, const uint32_t *__restrict__ cellT,
                                            int level_dense, int64_t seg_base, int64_t n_end, float box, float half,
                                            Cand *tile, uint32_t *rs, uint32_t *ro, int lane, uint32_t lt, F &&fn)
{
    const float eps = box * 9.5367431640625e-7f;   // 2^-20 of the box: far above coordinate rounding
    const int ncells = g.full ? 1 : g.nx * g.ny * g.nz;
    for (int cb = 0; cb < ncells; cb += 32) {
        uint32_t ra = 0, rb = 0;
        const int ci = cb + lane;
        if (g.full) {
            if (lane == 0) { ra = (uint32_t)seg_base; rb = (uint32_t)n_end; }
        } else if (ci < ncells) {
            const int ix = g.c0x + ci % g.nx, iy = g.c0y + (ci / g.nx) % g.ny, iz = g.c0z + ci / (g.nx * g.ny);
            bool keep = true;
            if (!g.pw) {
                const float gx = cg_gap(ix * g.csz, (ix + 1) * g.csz, g.flx, g.fhx, eps);
                const float gy = cg_gap(iy * g.csz, (iy + 1) * g.csz, g.fly, g.fhy, eps);
                const float gz = cg_gap(iz * g.csz, (iz + 1) * g.csz, g.flz, g.fhz, eps);
                keep = gx * gx + gy * gy + gz * gz <= g.r2c;
            }
            if (keep) {
                const int G = g.G;
                const int rx = ((ix % G) + G) % G, ry = ((iy % G) + G) % G, rz = ((iz % G) + G) % G;
                cell_range(cellT, keys, level_dense, g.l, morton3((uint32_t)rx, (uint32_t)ry, (uint32_t)rz), ra, rb);
            }
        }
        const uint32_t len = rb - ra;
        uint32_t inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kAll, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t total = __shfl_sync(kAll, inc, 31);
        __syncwarp();
        rs[lane] = ra;
        ro[lane] = inc - len;
        if (lane == 31) ro[32] = inc;
        __syncwarp();
        float4 pv[kCgPer];
        uint32_t pidx[kCgPer];
        int cur = 0;
        auto fetch = [&](uint32_t t0) {
#pragma unroll
            for (int jj = 0; jj < kCgPer; ++jj) {
                const uint32_t gi = t0 + (uint32_t)(lane + 32 * jj);
                pidx[jj] = 0xffffffffu;
                if (gi < total) {
                    while (ro[cur + 1] <= gi) ++cur;
                    pidx[jj] = rs[cur] + (gi - ro[cur]);
                }
            }
#pragma unroll
            for (int jj = 0; jj < kCgPer; ++jj)
                if (pidx[jj] != 0xffffffffu) pv[jj] = spos[pidx[jj]];
        };
        if (total > 0) fetch(0);
        for (uint32_t t0 = 0; t0 < total; t0 += kCgTile) {
            int m = 0;
#pragma unroll
            for (int jj = 0; jj < kCgPer; ++jj) {
                Cand c;
                bool keep = false;
                if (pidx[jj] != 0xffffffffu) {
                    const float4 v = pv[jj];
                    if (g.pw) {
                        c.x = v.x; c.y = v.y; c.z = v.z;
                        keep = true;
                    } else {
                        c.x = (g.wx && v.x >= half) ? v.x - box : v.x;
                        c.y = (g.wy && v.y >= half) ? v.y - box : v.y;
                        c.z = (g.wz && v.z >= half) ? v.z - box : v.z;
                        const float gx = cg_gap(c.x, c.x, g.flx, g.fhx, eps);
                        const float gy = cg_gap(c.y, c.y, g.fly, g.fhy, eps);
                        const float gz = cg_gap(c.z, c.z, g.flz, g.fhz, eps);
                        keep = gx * gx + gy * gy + gz * gz <= g.r2c;
                    }
                    c.s = pidx[jj];
                }
                const uint32_t kb = __ballot_sync(kAll, keep);
                if (keep) tile[m + __popc(kb & lt)] = c;
                m += __popc(kb);
            }
            // pad to a multiple of 32 with entries no test accepts
            if (lane < ((32 - (m & 31)) & 31)) {
                Cand z;
                z.x = z.y = z.z = __int_as_float(0x7fc00000);
                z.s = 0;
                tile[m + lane] = z;
            }
            __syncwarp();
            if (t0 + kCgTile < total) fetch(t0 + kCgTile);
            if (m > 0) fn(m);
            __syncwarp();
        }
    }
}

// d^2 of a staged candidate from the query: frame differences, or each
// pair's own minimum image (pw).
__device__ __forceinline__ float cand_d2(const Cand &c, bool pw, float qx, float qy, float qz, float rqx, float rqy,
                                         float rqz, float box, float half)
{
    float dx, dy, dz;
    if (pw) {
        dx = wrapdiff(c.x, rqx, box, half);
        dy = wrapdiff(c.y, rqy, box, half);
        dz = wrapdiff(c.z, rqz, box, half);
    } else {
        dx = c.x - qx;
        dy = c.y - qy;
        dz = c.z - qz;
    }
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// From the P histogram rows of each query group: the bin holding the rank-th
// entry (-1 if the rows hold fewer), the entries below that bin and up to
// it.  tot = all counted entries.  All lanes call it; results are uniform in
// each group.  Lane p of a group sums bins [p * PER, (p + 1) * PER) over the
// group's rows; a prefix over the group finds the lane holding the entry.
template <int P>
__device__ __forceinline__ void rows_find(const int *hist, int q, int p, int rank, int &bin, int &below, int &upto,
                                          int &tot)
{
    constexpr int PER = kBins / P;
    const int *h0 = hist + (p * PER) * 32 + q * P;
    int mine = 0;
#pragma unroll 4
    for (int i = 0; i < PER; ++i) {
#pragma unroll
        for (int r = 0; r < P; ++r) mine += h0[i * 32 + ((r + p) & (P - 1))];   // lanes p of a group: distinct banks
    }
    int incl = mine;
#pragma unroll
    for (int o = 1; o < P; o <<= 1) {
        const int y = __shfl_up_sync(kAll, incl, o, P);
        if (p >= o) incl += y;
    }
    const int excl = incl - mine;
    tot = __shfl_sync(kAll, incl, P - 1, P);
    int fb = 0, fbelow = 0, fupto = 0;
    if (excl < rank && rank <= incl) {
        int cum = excl;
        for (int i = 0; i < PER; ++i) {
            int h = 0;
#pragma unroll
            for (int r = 0; r < P; ++r) h += h0[i * 32 + ((r + p) & (P - 1))];
            if (cum + h >= rank) {
                fb = p * PER + i + 1;
                fbelow = cum;
                fupto = cum + h;
                break;
            }
            cum += h;
        }
    }
    bin = gsum<P>(fb) - 1;
    below = gsum<P>(fbelow);
    upto = gsum<P>(fupto);
}

// The rank-th smallest of a query's list entries above lo when more than
// kKC of them share its bin: a radix descent on the bit pattern of d^2 (4
// bits per level, a 16-bin histogram in h16 per level).  Kept out of line:
// crowded bins are rare, and the common path stays small.
template <int P>
__device__ __noinline__ float list_kth_deep(bool deep, const float *Ld, int cnt, int cmax, float lo, int below,
                                            int rank, int *h16, int p)
{
    uint32_t pfx = 0;
    int bel = below;
    for (int sh = 28; sh >= 0; sh -= 4) {
        __syncwarp();
        if (deep)
            for (int i = p; i < 16; i += P) h16[i] = 0;
        __syncwarp();
        for (int e0 = 0; e0 < cmax; e0 += P) {
            const int e = e0 + p;
            if (deep && e < cnt) {
                const float v = Ld[e];
                const uint32_t u = __float_as_uint(v);
                if (v > lo && (sh == 28 || (u >> (sh + 4)) == pfx)) atomicAdd(&h16[(u >> sh) & 15], 1);
            }
        }
        __syncwarp();
        if (deep) {
            int cum = bel, dsel = 15, dbel = bel;
            for (int i = 0; i < 16; ++i) {
                const int hh = h16[i];
                if (cum + hh >= rank) {
                    dsel = i;
                    dbel = cum;
                    break;
                }
                cum += hh;
            }
            pfx = (pfx << 4) | (uint32_t)dsel;
            bel = dbel;
        }
    }
    __syncwarp();
    return __uint_as_float(pfx);
}

// Exact rank-th smallest d^2 of a query's list: its entries in (lo, hi] are
// the bin holding it, with `below` smaller entries outside the bin.  Up to
// kKC entries are gathered and ranked; a larger bin goes through a radix
// descent on the bit pattern (4 bits per level).  All lanes call it with
// warp-uniform cmax; the result is uniform in each group.
template <int P>
__device__ float list_kth(bool member, const float *Ld, int cnt, int cmax, float lo, int below, int upto, int rank,
                          float *kd, int p, uint32_t gmask, uint32_t lt)
{
    const int mk = upto - below;
    float vk = -1.f;
    int nk = 0;
    for (int e0 = 0; e0 < cmax; e0 += P) {
        const int e = e0 + p;
        float v = 0.f;
        bool in = false;
        if (member && e < cnt) {
            v = Ld[e];
            in = v > lo;
        }
        const uint32_t bal = __ballot_sync(kAll, in);
        const int pos = nk + __popc(bal & gmask & lt);
        if (in && pos < kKC) kd[pos] = v;
        nk += __popc(bal & gmask);
    }
    __syncwarp();
    const bool small = mk <= kKC;
    const int mg = min(nk, kKC);   // equals mk: the list holds the bin's entries
    const int mkmax = cg_wmax_i((member && small) ? mg : 0);
    for (int e0 = 0; e0 < mkmax; e0 += P) {
        const int e = e0 + p;
        const bool mine = member && small && e < mg;
        const float v = mine ? kd[e] : 0.f;
        int l0 = below, le = below;
        for (int f = 0; f < mkmax; ++f) {
            if (f < mg) {
                const float u = kd[f];
                l0 += u < v;
                le += u <= v;
            }
        }
        if (mine && l0 < rank && rank <= le) vk = v;
    }
    if (__any_sync(kAll, member && !small)) {
        const float vd = list_kth_deep<P>(member && !small, Ld, cnt, cmax, lo, below, rank, (int *)kd, p);
        if (member && !small) vk = vd;
    }
    return gmaxf<P>(vk);
}

template <int P, bool SEG>
__global__ void __launch_bounds__(kCgWarps * 32, 4) knn_cg_kernel(CgDev a)
{
    constexpr int Q = 32 / P;
    using L = CgSmem<Q>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int q = lane / P, p = lane % P;
    const uint32_t gmask = (P == 32) ? kAll : (((1u << P) - 1u) << (q * P));
    const uint32_t lt = (1u << lane) - 1u;
    const int capq = a.capq;
    unsigned char *wb = smem_raw + L::total(capq) * wib;
    Cand *tile = (Cand *)(wb + L::tile);
    uint32_t *rs = (uint32_t *)(wb + L::rs);
    uint32_t *ro = (uint32_t *)(wb + L::ro);
    int *hist = (int *)(wb + L::uni);
    const int k = a.k;
    const int n_out = a.nbr_s ? a.n_out : 0;
    unsigned long long cand_acc = 0;
    uint32_t search_acc = 0, retry_acc = 0, warp_acc = 0;

    for (;;) {
        unsigned long long ch = 0;
        if (lane == 0) ch = atomicAdd(a.chunk_counter, 1ull);
        ch = __shfl_sync(kAll, ch, 0);
        if ((int64_t)ch >= a.n_chunks) break;
        ++warp_acc;
        int64_t s_first, n_end, seg_base;
        float box, half, inv_box, norm, plain_r;
        const uint32_t *cellT;
        int level_dense;
        if constexpr (SEG) {
            const SegDesc &sd = a.seg[seg_of_chunk(a.seg, a.B, (int64_t)ch)];
            seg_base = sd.base;
            n_end = sd.base + sd.n;
            s_first = sd.base + ((int64_t)ch - sd.chunk0) * Q;
            box = (float)sd.box;
            half = (float)(0.5 * sd.box);
            inv_box = (float)(1.0 / sd.box);
            norm = (float)sd.norm;
            cellT = a.cellT + sd.cell0;
            level_dense = sd.level_dense;
            plain_r = sd.plain_r;
        } else {
            seg_base = 0;
            n_end = a.n;
            s_first = (int64_t)ch * Q;
            box = a.box;
            half = a.half_box;
            inv_box = a.inv_box;
            norm = a.norm;
            cellT = a.cellT;
            level_dense = a.level_dense;
            plain_r = a.plain_r;
        }
        const int nq = (int)min((int64_t)Q, n_end - s_first);
        const bool active = q < nq;
        const int64_t sq = s_first + (active ? q : 0);
        const float4 qv = a.spos[sq];
        const float rqx = qv.x, rqy = qv.y, rqz = qv.z;
        float R0 = a.chunk_r ? a.chunk_r[ch] : plain_r;
        if (!(R0 > 0.f)) R0 = box * 1e-6f;
        // groups: a query farther than R0 from the one before it starts one
        const float px = __shfl_up_sync(kAll, rqx, P), py = __shfl_up_sync(kAll, rqy, P),
                    pz = __shfl_up_sync(kAll, rqz, P);
        const float ex = rqx - px, ey = rqy - py, ez = rqz - pz;
        const bool cut = q > 0 && active && ex * ex + ey * ey + ez * ez > R0 * R0;
        const uint32_t cutl = __ballot_sync(kAll, cut && p == 0);
        int g0 = 0;
        while (g0 < nq) {
            int g1 = g0 + 1;
            while (g1 < nq && !((cutl >> (g1 * P)) & 1u)) ++g1;
            const bool member = q >= g0 && q < g1;
            const int nmem = g1 - g0;
            g0 = g1;

            // ------------- count passes.  First until every member holds
            // Ndens entries within R (certified), then, for members whose
            // list up to the Ndens-th bin would not fit, again in a finer
            // (or lower) window of that bin.
            float R = R0;
            int tries = 0, refines = 0;
            bool certified = false, failed = false;
            Region rg = make_region(member, rqx, rqy, rqz, R, box, half, inv_box, a.cpr);
            int top = (int)(__float_as_uint(rg.full ? 0.76f * box * box : R * R) >> kShift0);
            int shift = kShift0, top0 = top;
            float tauA = rg.full ? INFINITY : R * R;
            bool counting = member;
            int bk = -1, below_k = 0, upto_k = 0, bk0 = -1, bo = -1, upto_o = 0;
            float edge_o = -1.f;
            for (;;) {
                ++search_acc;
                if (counting) {
#pragma unroll 8
                    for (int b = 0; b < kBins; ++b) hist[b * 32 + lane] = 0;
                }
                __syncwarp();
                {
                    const float qx = (!rg.pw && rg.wx && rqx >= half) ? rqx - box : rqx;
                    const float qy = (!rg.pw && rg.wy && rqy >= half) ? rqy - box : rqy;
                    const float qz = (!rg.pw && rg.wz && rqz >= half) ? rqz - box : rqz;
                    const int base = top - (kBins - 1);
                    int *hcol = hist + lane;
                    scan_region(rg, a.spos, a.keys, cellT, level_dense, seg_base, n_end, box, half, tile, rs, ro,
                                lane, lt, [&](int m) {
                                    cand_acc += (unsigned long long)m * (unsigned long long)nmem;
                                    if (counting) {
                                        for (int j = p; j < m; j += P) {
                                            const float d2 =
                                                cand_d2(tile[j], rg.pw, qx, qy, qz, rqx, rqy, rqz, box, half);
                                            if (d2 <= tauA) {
                                                const int b = max((int)(__float_as_uint(d2) >> shift) - base, 0);
                                                hcol[b * 32] += 1;
                                            }
                                        }
                                    }
                                });
                }
                __syncwarp();
                int nbk, nbel, nup, ntot;
                rows_find<P>(hist, q, p, k, nbk, nbel, nup, ntot);
                if (counting) {
                    bk = nbk;
                    below_k = nbel;
                    upto_k = nup;
                }
                if (!certified) {
                    const bool ok = !member || ntot >= k;
                    if (!__all_sync(kAll, ok)) {
                        ++retry_acc;
                        if (++tries >= kCgTries || rg.full) {
                            if (lane == 0) atomicOr(a.err, kErrKnnRetry);
                            failed = true;
                            break;
                        }
                        float f = 1.25f;
                        if (!ok) f = fmaxf(f, 1.1f * cbrtf((float)k / (float)max(ntot, 1)));
                        f = cg_wmax(f);
                        R *= fminf(f, 8.f);
                        rg = make_region(member, rqx, rqy, rqz, R, box, half, inv_box, a.cpr);
                        top = top0 = (int)(__float_as_uint(rg.full ? 0.76f * box * box : R * R) >> kShift0);
                        tauA = rg.full ? INFINITY : R * R;
                        continue;
                    }
                    certified = true;
                    bk0 = bk;
                    if (n_out > 0) {
                        int b2, t2;
                        rows_find<P>(hist, q, p, n_out, bo, b2, upto_o, t2);
                        edge_o = bin_edge(top - (kBins - 1), shift, bo);
                    }
                }
                // the list up to the Ndens-th bin must fit: refine crowded bins
                counting = member && upto_k > capq;
                if (!__any_sync(kAll, counting)) break;
                if (++refines > kRefine) {
                    if (lane == 0) atomicOr(a.err, kErrDegenerate);
                    failed = true;
                    break;
                }
                if (counting) {
                    const int base = top - (kBins - 1);
                    if (bk == 0 && base > 0) {
                        // the Ndens-th entry lies in the open lowest bin: move the window down
                        tauA = fminf(tauA, bin_edge(base, shift, 0));
                        top -= kBins - 1;
                    } else if (shift > 0) {
                        // 64 finer bins of bin bk
                        const int ns = max(shift - 6, 0), d = shift - ns;
                        tauA = fminf(tauA, bin_edge(base, shift, bk));
                        top = ((base + bk) << d) | ((1 << d) - 1);
                        shift = ns;
                    } else {
                        // every entry of the bin has the same d^2: more ties
                        // than the list holds
                        if (p == 0) atomicOr(a.err, kErrDegenerate);
                        failed = true;
                    }
                }
                if (__any_sync(kAll, failed)) break;
            }
            if (failed) continue;
            const int base = top - (kBins - 1);
            const float edge_k = fminf(bin_edge(base, shift, bk), rg.full ? INFINITY : R * R);
            const float lo_k = bk > 0 ? bin_edge(base, shift, bk - 1) : -1.f;
            if ((shift != kShift0 || top != top0) && bo >= bk0) {
                // refined: the n_out-th entry keeps its first-window bin only
                // when that bin lies below the refined one
                edge_o = edge_k;
                upto_o = upto_k;
            }
            edge_o = fminf(edge_o, edge_k);

            // ------------- scan B: gather every entry up to the Ndens-th bin
            if (!rg.full) {
                const float rB = sqrtf(cg_wmax(member ? edge_k : 0.f)) * 1.00001f;
                rg = make_region(member, rqx, rqy, rqz, fminf(R, rB), box, half, inv_box, a.cpr);
            }
            float *Ld = (float *)(hist) + q * capq;                                // this query's list: d^2 ...
            uint32_t *Ls = (uint32_t *)(wb + L::ls(capq)) + q * capq;              // ... and sorted index
            int cnt = 0;
            {
                const float qx = (!rg.pw && rg.wx && rqx >= half) ? rqx - box : rqx;
                const float qy = (!rg.pw && rg.wy && rqy >= half) ? rqy - box : rqy;
                const float qz = (!rg.pw && rg.wz && rqz >= half) ? rqz - box : rqz;
                scan_region(rg, a.spos, a.keys, cellT, level_dense, seg_base, n_end, box, half, tile, rs, ro, lane,
                            lt, [&](int m) {
                                cand_acc += (unsigned long long)m * (unsigned long long)nmem;
                                for (int j0 = 0; j0 < m; j0 += P) {
                                    const Cand c = tile[j0 + p];
                                    const float d2 = cand_d2(c, rg.pw, qx, qy, qz, rqx, rqy, rqz, box, half);
                                    const bool keep = member && d2 <= edge_k;
                                    const uint32_t bal = __ballot_sync(kAll, keep);
                                    const int pos = cnt + __popc(bal & gmask & lt);
                                    if (keep && pos < capq) {
                                        Ld[pos] = d2;
                                        Ls[pos] = c.s;
                                    }
                                    cnt += __popc(bal & gmask);
                                }
                            });
            }
            __syncwarp();
            if (__any_sync(kAll, member && cnt != upto_k)) {
                // the two scans disagree: cannot happen with exact arithmetic
                if (lane == 0) atomicOr(a.err, kErrKnnRetry);
                continue;
            }

            // ------------- selection
            float *kd = (float *)(wb + L::kd(capq)) + q * kKC;
            float *od = (float *)(wb + L::od(capq)) + q * kOC;
            uint32_t *os = (uint32_t *)(wb + L::os(capq)) + q * kOC;
            const int cmax = cg_wmax_i(member ? cnt : 0);
            // (1) the exact Ndens-th d^2
            const float vk = list_kth<P>(member, Ld, cnt, cmax, lo_k, below_k, upto_k, k, kd, p, gmask, lt);
            // (2) density: fixed-point sum of w(2 r / r_k) over entries with d^2 < r_k^2
            unsigned long long wsum = 0;
            const float rk = sqrtf(vk);
            const float inv_h = vk > 0.f ? 2.f / rk : 0.f;
            for (int e0 = 0; e0 < cmax; e0 += P) {
                const int e = e0 + p;
                if (member && e < cnt) {
                    const float v = Ld[e];
                    if (v < vk) {
                        const float w = m4<float>(sqrtf(v) * inv_h);
                        wsum += (unsigned long long)(w * 4294967296.0f + 0.5f);
                    }
                }
            }
#pragma unroll
            for (int o = 1; o < P; o <<= 1) wsum += __shfl_xor_sync(kAll, wsum, o);
            // (3) the n_out nearest in (d^2, original index) order
            if (n_out > 0) {
                const bool small = upto_o <= kOC;
                if (__any_sync(kAll, member && small)) {
                    int no = 0;
                    for (int e0 = 0; e0 < cmax; e0 += P) {
                        const int e = e0 + p;
                        float v = 0.f;
                        uint32_t sv = 0;
                        bool in = false;
                        if (member && small && e < cnt) {
                            v = Ld[e];
                            sv = Ls[e];
                            in = v <= edge_o;
                        }
                        const uint32_t bal = __ballot_sync(kAll, in);
                        const int pos = no + __popc(bal & gmask & lt);
                        if (in && pos < kOC) {
                            od[pos] = v;
                            os[pos] = sv;
                        }
                        no += __popc(bal & gmask);
                    }
                    __syncwarp();
                    // only gathered entries are read (no equals upto_o)
                    const int ng = min(no, kOC);
                    const int nomax = cg_wmax_i((member && small) ? ng : 0);
                    for (int e0 = 0; e0 < nomax; e0 += P) {
                        const int e = e0 + p;
                        const bool mine = member && small && e < ng;
                        const float v = mine ? od[e] : 0.f;
                        const uint32_t se = mine ? os[e] : 0u;
                        uint32_t oe = 0xffffffffu;
                        int rank = 0;
                        for (int f = 0; f < nomax; ++f) {
                            if (f < ng) {
                                const float u = od[f];
                                rank += u < v;
                                if (mine && u == v && f != e) {
                                    if (oe == 0xffffffffu) oe = __float_as_uint(a.spos[se].w);
                                    rank += __float_as_uint(a.spos[os[f]].w) < oe;
                                }
                            }
                        }
                        if (mine && rank < n_out) a.nbr_s[(size_t)sq * a.ld_out + rank] = se;
                    }
                }
                if (__any_sync(kAll, member && !small)) {
                    // many entries up to the n_out-th bin: rank in the list itself
                    for (int e0 = 0; e0 < cmax; e0 += P) {
                        const int e = e0 + p;
                        if (!(member && !small && e < cnt)) continue;
                        const float v = Ld[e];
                        if (!(v <= edge_o)) continue;
                        const uint32_t se = Ls[e];
                        uint32_t oe = 0xffffffffu;
                        int rank = 0;
                        for (int f = 0; f < cnt; ++f) {
                            const float u = Ld[f];
                            if (u < v) {
                                ++rank;
                                continue;
                            }
                            if (u == v && f != e) {
                                if (oe == 0xffffffffu) oe = __float_as_uint(a.spos[se].w);
                                rank += __float_as_uint(a.spos[Ls[f]].w) < oe;
                            }
                        }
                        if (rank < n_out) a.nbr_s[(size_t)sq * a.ld_out + rank] = se;
                    }
                }
            }
            if (member && p == 0) {
                float dens;
                if (vk > 0.f) {
                    const float h = rk * 0.5f;
                    dens = (float)(norm * ((float)wsum * 2.3283064365386963e-10f) / (h * h * h));
                } else {
                    dens = INFINITY;
                }
                a.dens_s[sq] = dens;
                if (a.rk_s) a.rk_s[sq] = rk;
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        atomicAdd(&a.counters[kCntCand], cand_acc);
        atomicAdd(&a.counters[kCntSearch], (unsigned long long)search_acc);
        atomicAdd(&a.counters[kCntRetry], (unsigned long long)retry_acc);
        atomicAdd(&a.counters[kCntWarps], (unsigned long long)warp_acc);
    }
}

// ======================================================= one query per warp
// The same count-then-gather search with the whole warp on one query.  A
// warp takes a chunk of kWqChunk consecutive particles (whose first radius
// comes from the radius of that chunk) and serves them one after another.
// For each query the warp lists the cells (side >= R / cpr, cpr <= 3) that
// meet its ball, and the lanes read the cells' particles straight from the
// sorted array -- 32 consecutive particles per step, no shared-memory
// staging -- with their own histogram rows (32 quarter-octave bins).  The
// list, the exact Ndens-th distance, the density and the n_out nearest
// follow as in the grouped kernel above.
constexpr int kWqChunk = 4;                 // queries per chunk (the radius is per chunk)
constexpr int kWqBins = 16;                 // histogram bins per lane row (quarter octaves of d^2)
constexpr int kWqBinsLog = 4;
constexpr int kWqGather = 320;              // entries the count scan keeps, so the gather scan can be skipped
constexpr int kWqCells = 128;               // cells of one query's region held at once

// Shared memory of one warp, byte offsets.  The histogram rows (count
// scans) share their space with the small selection lists (kd, od, os);
// the count scan's list (gd, gs: kWqGather entries) shares its space with
// the gather scan's list (Ld, Ls: capq entries), which is only used when
// the first is too short.
struct WqSmem {
    static constexpr size_t cra = 0;                                   // kWqCells range starts
    static constexpr size_t cln = cra + kWqCells * 4;                  // kWqCells range lengths
    static constexpr size_t cmd = cln + kWqCells * 4;                  // kWqCells min distance^2 to the query
    static constexpr size_t cpre = cmd + kWqCells * 4;                 // kWqCells + 1 prefix offsets
    static constexpr size_t hist = (cpre + (kWqCells + 1) * 4 + 15) & ~size_t(15);
    static constexpr size_t hist_bytes = (size_t)kWqBins * 32 * 4;
    static constexpr size_t kd = hist;
    static constexpr size_t od = kd + kKC * 4;
    static constexpr size_t os = od + kOC * 4;
    static_assert(kKC * 4 + kOC * 8 <= hist_bytes, "selection lists fit the histogram rows");
    static constexpr size_t gd = hist + hist_bytes;
    static constexpr size_t gs = gd + kWqGather * 4;
    __host__ __device__ static size_t ls(int capq) { return gd + (size_t)capq * 4; }
    __host__ __device__ static size_t total(int capq)
    {
        const size_t g = kWqGather * 8 > (size_t)capq * 8 ? kWqGather * 8 : (size_t)capq * 8;
        return (gd + g + 15) & ~size_t(15);
    }
};

// Per-bin totals of the histogram rows (lane b < kWqBins: bin b, summed by
// lanes b and b + 16 over half the columns each; column c of row b is read
// at (c + b) mod 32, so every load hits 32 banks) and their inclusive prefix
// over the lanes; tot = all counted entries.  Uniform over the warp.
__device__ __forceinline__ void wq_rows_prefix(const int *hist, int lane, int &mine, int &incl, int &tot)
{
    static_assert(kWqBins == 16, "two lanes per histogram row");
    const int row = lane & 15, c0 = (lane >> 4) * 16;
    int part = 0;
#pragma unroll 8
    for (int r = 0; r < 16; ++r) part += hist[row * 32 + ((c0 + r + row) & 31)];
    part += __shfl_xor_sync(kAll, part, 16);
    mine = lane < kWqBins ? part : 0;
    incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kAll, incl, o);
        if (lane >= o) incl += y;
    }
    tot = __shfl_sync(kAll, incl, 31);
}

// The bin holding the rank-th entry (-1 if fewer entries), the entries below
// it and up to it, from the per-bin totals and prefix.
__device__ __forceinline__ void wq_rows_rank(int mine, int incl, int rank, int &bin, int &below, int &upto)
{
    const uint32_t hit = __ballot_sync(kAll, incl - mine < rank && rank <= incl);
    const int l = hit ? __ffs(hit) - 1 : 0;
    bin = hit ? l : -1;
    below = __shfl_sync(kAll, incl - mine, l);
    upto = __shfl_sync(kAll, incl, l);
}

// Lists the non-empty cells of level l (frame coordinates) within r of the
// query; returns their count, or -1 if more than kWqCells meet the ball.
__device__ int wq_cells(float qx, float qy, float qz, float r, float box, float inv_box, int l,
                        const uint32_t *__restrict__ cellT, const uint64_t *__restrict__ keys, int level_dense,
                        uint32_t *cra, uint32_t *cln, float *cmd, int lane, uint32_t lt)
{
    const int G = 1 << l;
    const float sc = inv_box * (float)G, csz = box / (float)G;
    const float eps = box * 9.5367431640625e-7f;
    const float r2c = r * r * 1.00001f + box * box * 1e-12f;
    int c0x = (int)floorf((qx - r) * sc), c0y = (int)floorf((qy - r) * sc), c0z = (int)floorf((qz - r) * sc);
    int nx = (int)floorf((qx + r) * sc) - c0x + 1, ny = (int)floorf((qy + r) * sc) - c0y + 1,
        nz = (int)floorf((qz + r) * sc) - c0z + 1;
    if (nx >= G) { c0x = 0; nx = G; }
    if (ny >= G) { c0y = 0; ny = G; }
    if (nz >= G) { c0z = 0; nz = G; }
    const int ncube = nx * ny * nz;
    // cell ci of the cube is (ci mod nx, (ci / nx) mod ny, ci / (nx ny)); the
    // quotients come from float reciprocals, exact for these small integers
    const float inx = 1.f / (float)nx, inxy = 1.f / (float)(nx * ny);
    int nkeep = 0;
    for (int cb = 0; cb < ncube; cb += 32) {
        const int ci = cb + lane;
        bool keep = false;
        uint32_t ra = 0, rb = 0;
        float md2 = 0.f;
        if (ci < ncube) {
            const int cz = (int)(((float)ci + 0.5f) * inxy);
            const int rxy = ci - cz * nx * ny;
            const int cy = (int)(((float)rxy + 0.5f) * inx);
            const int ix = c0x + (rxy - cy * nx), iy = c0y + cy, iz = c0z + cz;
            const float gx = cg_gap(qx, qx, ix * csz, (ix + 1) * csz, eps);
            const float gy = cg_gap(qy, qy, iy * csz, (iy + 1) * csz, eps);
            const float gz = cg_gap(qz, qz, iz * csz, (iz + 1) * csz, eps);
            md2 = gx * gx + gy * gy + gz * gz;
            if (md2 <= r2c) {
                cell_range(cellT, keys, level_dense, l,
                           morton3((uint32_t)(ix & (G - 1)), (uint32_t)(iy & (G - 1)), (uint32_t)(iz & (G - 1))), ra,
                           rb);
                keep = rb > ra;
            }
        }
        const uint32_t bal = __ballot_sync(kAll, keep);
        const int pos = nkeep + __popc(bal & lt);
        if (keep && pos < kWqCells) {
            cra[pos] = ra;
            cln[pos] = rb - ra;
            cmd[pos] = md2;
        }
        nkeep += __popc(bal);
    }
    __syncwarp();
    return nkeep <= kWqCells ? nkeep : -1;
}

// Exclusive prefix of the nc cell lengths into cpre[0..nc]; returns the total.
__device__ __forceinline__ uint32_t wq_prefix(const uint32_t *cln, uint32_t *cpre, int nc, int lane)
{
    constexpr int PER = kWqCells / 32;
    static_assert(PER == 4, "one 16-byte read of cell lengths per lane");
    uint4 q = make_uint4(0u, 0u, 0u, 0u);
    if (lane * PER < nc) q = reinterpret_cast<const uint4 *>(cln)[lane];
    const uint32_t v[PER] = {nc > lane * PER ? q.x : 0u, nc > lane * PER + 1 ? q.y : 0u,
                             nc > lane * PER + 2 ? q.z : 0u, nc > lane * PER + 3 ? q.w : 0u};
    const uint32_t mine = v[0] + v[1] + v[2] + v[3];
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kAll, incl, o);
        if (lane >= o) incl += y;
    }
    uint32_t run = incl - mine;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int j = lane * PER + i;
        if (j < nc) cpre[j] = run;
        run += v[i];
    }
    const uint32_t total = __shfl_sync(kAll, incl, 31);
    if (lane == 0) cpre[nc] = total;
    __syncwarp();
    return total;
}

// Visits the particles of cells [0, nc) (ranges cra/cln, prefix cpre), 32
// consecutive ones per step, lane t taking particle g0 + t: fn(v, s, valid).
// The cell of each lane's particle comes from the cell starts inside the
// step's window (one bit each), so no lane searches the prefix.  (Issuing
// several steps' loads ahead measured slower: the larger loop body costs
// more in instruction fetch and registers than the overlap gains.)
template <typename F>
__device__ __forceinline__ void wq_visit(const float4 *__restrict__ spos, const uint32_t *cra, const uint32_t *cpre,
                                         int nc, uint32_t total, int lane, F &&fn)
{
    constexpr int U = 1;
    int cbase = -1;   // the cell holding particle g0 - 1
    const uint32_t upto_lane = lane == 31 ? kAll : ((2u << lane) - 1u);
    for (uint32_t g0 = 0; g0 < total; g0 += 32 * U) {
        uint32_t s[U];
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t w0 = g0 + 32 * u;
            const int j = cbase + 1 + lane;
            const uint32_t st = j < nc ? cpre[j] : total;
            const uint32_t bit = (st >= w0 && st < w0 + 32) ? 1u << (st - w0) : 0u;
            const uint32_t starts = __reduce_or_sync(kAll, bit);
            const int c = cbase + __popc(starts & upto_lane);
            const uint32_t g = w0 + (uint32_t)lane;
            s[u] = g < total ? cra[c] + (g - cpre[c]) : 0xffffffffu;
            cbase += __popc(starts);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (s[u] != 0xffffffffu) v[u] = spos[s[u]];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) fn(v[u], s[u], s[u] != 0xffffffffu);
    }
}

// The n_out nearest of a warp's list when more than kOC entries lie up to
// the n_out-th bin (long Nhop lists, ties): each entry up to edge_o is
// ranked by (d^2, original index) against the whole list.  A lane ranks
// four entries (e, e + 32, e + 64, e + 96) in one pass over the list.  The
// first pass counts smaller distances only and writes the row; the ranks
// of the m entries are then 0 .. m-1, summing to m(m-1)/2, unless two
// distances are equal.  Only then does a second pass rank again by
// (d^2, original index) and overwrite every position the first one wrote.
// Out of line: the common path gathers at most kOC entries instead.
__device__ __noinline__ void wq_rank_in_list(const float *Ld, const uint32_t *Ls, int cnt, float edge_o, int n_out,
                                             const float4 *__restrict__ spos, uint32_t *row, int lane)
{
    constexpr int B = 4;
    int m = 0, sum = 0;
    for (int e0 = 0; e0 < cnt; e0 += 32 * B) {
        float v[B];
        int rank[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int e = e0 + 32 * j + lane;
            v[j] = e < cnt ? Ld[e] : INFINITY;
            if (!(v[j] <= edge_o)) v[j] = -1.f;   // not ranked; compares as nothing below it
            rank[j] = 0;
        }
        for (int f = 0; f < cnt; ++f) {
            const float u = Ld[f];
#pragma unroll
            for (int j = 0; j < B; ++j) rank[j] += u < v[j];
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
            if (!(v[j] >= 0.f)) continue;
            ++m;
            sum += rank[j];
            if (rank[j] < n_out) row[rank[j]] = Ls[e0 + 32 * j + lane];
        }
    }
    m = (int)__reduce_add_sync(kAll, (unsigned)m);
    sum = (int)__reduce_add_sync(kAll, (unsigned)sum);
    if (sum == m * (m - 1) / 2) return;
    __syncwarp();
    for (int e0 = 0; e0 < cnt; e0 += 32 * B) {
        float v[B];
        int rank[B];
        uint32_t oe[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int e = e0 + 32 * j + lane;
            v[j] = e < cnt ? Ld[e] : INFINITY;
            if (!(v[j] <= edge_o)) v[j] = -1.f;
            rank[j] = 0;
            oe[j] = v[j] >= 0.f ? __float_as_uint(spos[Ls[e]].w) : 0u;
        }
        for (int f = 0; f < cnt; ++f) {
            const float u = Ld[f];
            bool tie = false;
#pragma unroll
            for (int j = 0; j < B; ++j) {
                rank[j] += u < v[j];
                tie |= u == v[j];
            }
            if (tie) {
                // the entry itself compares equal, never below
                const uint32_t of = __float_as_uint(spos[Ls[f]].w);
#pragma unroll
                for (int j = 0; j < B; ++j) rank[j] += u == v[j] && of < oe[j];
            }
        }
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (v[j] >= 0.f && rank[j] < n_out) row[rank[j]] = Ls[e0 + 32 * j + lane];
    }
}

// Bitonic sort across the warp, one element per lane, ascending by lane.
__device__ __forceinline__ float warp_sort32(float v, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const float o = __shfl_xor_sync(kAll, v, j);
            v = (((lane & j) == 0) == ((lane & k) == 0)) ? fminf(v, o) : fmaxf(v, o);
        }
    }
    return v;
}

__device__ __forceinline__ void warp_sort32(unsigned long long &key, uint32_t &pay, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(kAll, key, j);
            const uint32_t op = __shfl_xor_sync(kAll, pay, j);
            const bool take = (((lane & j) == 0) == ((lane & k) == 0)) ? o < key : o > key;
            if (take) {
                key = o;
                pay = op;
            }
        }
    }
}

// The same for a float key with a payload (equal keys in any order).
__device__ __forceinline__ void warp_sort32_kv(float &key, uint32_t &pay, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const float o = __shfl_xor_sync(kAll, key, j);
            const uint32_t op = __shfl_xor_sync(kAll, pay, j);
            const bool take = (((lane & j) == 0) == ((lane & k) == 0)) ? o < key : o > key;
            if (take) {
                key = o;
                pay = op;
            }
        }
    }
}

// The payloads of a warp sort by (d^2 bits, original index): the n_out list
// when two distances are equal.  Out of line: it is rare.
__device__ __noinline__ uint32_t wq_tie_sort(unsigned long long key, uint32_t pay, int lane)
{
    warp_sort32(key, pay, lane);
    return pay;
}

// Exact rank-th smallest d^2 of the warp's list, whose entries in (lo, ...]
// hold it with `below` smaller entries outside: up to 32 such entries (the
// k-th bin) are sorted across the warp; more go through the radix descent.
__device__ __forceinline__ float wq_list_kth(const float *Ld, int cnt, float lo, int below, int upto, int rank,
                                             float *kd, int lane, uint32_t lt)
{
    if (upto - below > 32)
        return list_kth_deep<32>(true, Ld, cnt, cnt, lo, below, rank, (int *)kd, lane);
    int nk = 0;
    for (int e0 = 0; e0 < cnt; e0 += 32) {
        const int e = e0 + lane;
        const float v = e < cnt ? Ld[e] : 0.f;
        const bool in = e < cnt && v > lo;
        const uint32_t bal = __ballot_sync(kAll, in);
        const int pos = nk + __popc(bal & lt);
        if (in && pos < 32) kd[pos] = v;
        nk += __popc(bal);
    }
    __syncwarp();
    const float mine = lane < nk ? kd[lane] : INFINITY;
    const float sorted = warp_sort32(mine, lane);
    return __shfl_sync(kAll, sorted, rank - below - 1);
}

template <bool SEG>
__global__ void __launch_bounds__(kCgWarps * 32, 8) knn_wq_kernel(CgDev a)
{
    using L = WqSmem;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int capq = a.capq;
    unsigned char *wb = smem_raw + L::total(capq) * wib;
    uint32_t *cra = (uint32_t *)(wb + L::cra);
    uint32_t *cln = (uint32_t *)(wb + L::cln);
    float *cmd = (float *)(wb + L::cmd);
    uint32_t *cpre = (uint32_t *)(wb + L::cpre);
    int *hist = (int *)(wb + L::hist);
    float *gd = (float *)(wb + L::gd);
    uint32_t *gs = (uint32_t *)(wb + L::gs);
    float *kd = (float *)(wb + L::kd);
    float *od = (float *)(wb + L::od);
    uint32_t *os = (uint32_t *)(wb + L::os);
    const int k = a.k;
    const int n_out = a.nbr_s ? a.n_out : 0;
    const int cpr = min(max(a.cpr, 1), 3);
    unsigned long long cand_acc = 0;
    uint32_t search_acc = 0, retry_acc = 0, warp_acc = 0;

    for (;;) {
        unsigned long long ch = 0;
        if (lane == 0) ch = atomicAdd(a.chunk_counter, 1ull);
        ch = __shfl_sync(kAll, ch, 0);
        if ((int64_t)ch >= a.n_chunks) break;
        ++warp_acc;
        int64_t s_first, n_end, seg_base;
        float box, half, inv_box, norm, plain_r;
        const uint32_t *cellT;
        int level_dense;
        if constexpr (SEG) {
            const SegDesc &sd = a.seg[seg_of_chunk(a.seg, a.B, (int64_t)ch)];
            seg_base = sd.base;
            n_end = sd.base + sd.n;
            s_first = sd.base + ((int64_t)ch - sd.chunk0) * kWqChunk;
            box = (float)sd.box;
            half = (float)(0.5 * sd.box);
            inv_box = (float)(1.0 / sd.box);
            norm = (float)sd.norm;
            cellT = a.cellT + sd.cell0;
            level_dense = sd.level_dense;
            plain_r = sd.plain_r;
        } else {
            seg_base = 0;
            n_end = a.n;
            s_first = (int64_t)ch * kWqChunk;
            box = a.box;
            half = a.half_box;
            inv_box = a.inv_box;
            norm = a.norm;
            cellT = a.cellT;
            level_dense = a.level_dense;
            plain_r = a.plain_r;
        }
        const int nq = (int)min((int64_t)kWqChunk, n_end - s_first);
        float R0 = a.chunk_r ? a.chunk_r[ch] : plain_r;
        if (!(R0 > 0.f)) R0 = box * 1e-6f;
        for (int qi = 0; qi < nq; ++qi) {
            const int64_t sq = s_first + qi;
            const float4 qv = a.spos[sq];
            const float rqx = qv.x, rqy = qv.y, rqz = qv.z;
            // ------------- count passes (certify, then refine a crowded bin)
            float R = R0;
            int tries = 0, refines = 0;
            bool certified = false, failed = false, full = false;
            float qx = rqx, qy = rqy, qz = rqz;
            bool fx = false, fy = false, fz = false;   // frame shift per axis
            bool shifted = false;                      // any of them (warp-uniform)
            int nc = 0, l = 1;
            uint32_t total = 0;
            int top = 0, shift = kShift0, top0 = 0;
            float tauA = 0.f;
            int bk = -1, below_k = 0, upto_k = 0, bk0 = -1, bo = -1, upto_o = 0;
            float edge_o = -1.f;
            bool fresh = true;   // the region must be (re)built for R
            int gn = 0;          // entries within R kept by the certifying count scan
            for (;;) {
                if (fresh) {
                    ++search_acc;
                    full = 2.f * R >= half;
                    // frame: on an axis where the ball crosses a face, coordinates
                    // >= L/2 move by -L (exact); a whole-box scan takes each
                    // pair's own minimum image
                    fx = !full && (rqx - R < 0.f || rqx + R >= box);
                    fy = !full && (rqy - R < 0.f || rqy + R >= box);
                    fz = !full && (rqz - R < 0.f || rqz + R >= box);
                    qx = (fx && rqx >= half) ? rqx - box : rqx;
                    qy = (fy && rqy >= half) ? rqy - box : rqy;
                    qz = (fz && rqz >= half) ? rqz - box : rqz;
                    shifted = fx || fy || fz;
                    if (full) {
                        if (lane == 0) {
                            cra[0] = (uint32_t)seg_base;
                            cln[0] = (uint32_t)(n_end - seg_base);
                            cmd[0] = 0.f;
                        }
                        __syncwarp();
                        nc = 1;
                    } else {
                        // the finest level with 2^l <= cells (side >= R / cpr), at
                        // least 1: floor(log2(cells)) is the float's exponent
                        const float cells = box * (float)cpr / R;
                        l = min(max((int)((__float_as_uint(cells) >> 23) & 0xFFu) - 127, 1), kMaxLevel);
                        for (;;) {
                            nc = wq_cells(qx, qy, qz, R, box, inv_box, l, cellT, a.keys, level_dense, cra, cln, cmd,
                                          lane, lt);
                            if (nc >= 0 || l <= 1) break;
                            --l;   // too many cells meet the ball: take coarser ones
                        }
                    }
                    total = wq_prefix(cln, cpre, nc, lane);
                    top = top0 = (int)(__float_as_uint(full ? 0.76f * box * box : R * R) >> kShift0);
                    shift = kShift0;
                    tauA = full ? INFINITY : R * R;
                    fresh = false;
                }
#pragma unroll
                for (int i = 0; i < kWqBins * 32 / 128; ++i)   // the rows, four words per lane per store
                    reinterpret_cast<int4 *>(hist)[i * 32 + lane] = make_int4(0, 0, 0, 0);
                __syncwarp();
                {
                    const int base = top - (kWqBins - 1);
                    int *hcol = hist + lane;
                    cand_acc += total;
                    // until certified, the particles within R are also kept
                    // (up to kWqGather), which spares the gather scan
                    const bool keep_list = !certified;
                    if (keep_list) gn = 0;
                    wq_visit(a.spos, cra, cpre, nc, total, lane, [&](const float4 &v, uint32_t s, bool valid) {
                        float dx = 0.f, dy = 0.f, dz = 0.f;
                        if (full) {
                            dx = wrapdiff(v.x, rqx, box, half);
                            dy = wrapdiff(v.y, rqy, box, half);
                            dz = wrapdiff(v.z, rqz, box, half);
                        } else if (shifted) {
                            dx = (fx && v.x >= half ? v.x - box : v.x) - qx;
                            dy = (fy && v.y >= half ? v.y - box : v.y) - qy;
                            dz = (fz && v.z >= half ? v.z - box : v.z) - qz;
                        } else {
                            dx = v.x - qx;
                            dy = v.y - qy;
                            dz = v.z - qz;
                        }
                        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        const bool in = valid && d2 <= tauA;
                        if (in) {
                            const int b = max((int)(__float_as_uint(d2) >> shift) - base, 0);
                            hcol[b * 32] += 1;
                        }
                        if (keep_list) {
                            const uint32_t bal = __ballot_sync(kAll, in);
                            const int pos = gn + __popc(bal & lt);
                            if (in && pos < kWqGather) {
                                gd[pos] = d2;
                                gs[pos] = s;
                            }
                            gn += __popc(bal);
                        }
                    });
                }
                __syncwarp();
                int ntot;
                int rmine, rincl;
                wq_rows_prefix(hist, lane, rmine, rincl, ntot);
                wq_rows_rank(rmine, rincl, k, bk, below_k, upto_k);
                if (!certified) {
                    if (ntot < k) {
                        ++retry_acc;
                        if (++tries >= kCgTries || full) {
                            if (lane == 0) atomicOr(a.err, kErrKnnRetry);
                            failed = true;
                            break;
                        }
                        R *= fminf(fmaxf(1.25f, 1.1f * cbrtf((float)k / (float)max(ntot, 1))), 8.f);
                        fresh = true;
                        continue;
                    }
                    certified = true;
                    bk0 = bk;
                    if (n_out > 0) {
                        int b2;
                        wq_rows_rank(rmine, rincl, n_out, bo, b2, upto_o);
                        edge_o = bin_edge(top - (kWqBins - 1), shift, bo);
                    }
                }
                // a complete list of the particles within R: the gather scan
                // is not needed, nor a finer count of a crowded bin
                if (gn <= kWqGather || upto_k <= capq) break;
                // a crowded Ndens-th bin: count again in a finer (or lower) window
                if (++refines > kRefine) {
                    if (lane == 0) atomicOr(a.err, kErrDegenerate);
                    failed = true;
                    break;
                }
                const int base = top - (kWqBins - 1);
                if (bk == 0 && base > 0) {
                    tauA = fminf(tauA, bin_edge(base, shift, 0));
                    top -= kWqBins - 1;
                } else if (shift > 0) {
                    const int ns = max(shift - kWqBinsLog, 0), d = shift - ns;
                    tauA = fminf(tauA, bin_edge(base, shift, bk));
                    top = ((base + bk) << d) | ((1 << d) - 1);
                    shift = ns;
                } else {
                    if (lane == 0) atomicOr(a.err, kErrDegenerate);
                    failed = true;
                    break;
                }
            }
            if (failed) continue;
            const int base = top - (kWqBins - 1);
            const float edge_k = fminf(bin_edge(base, shift, bk), full ? INFINITY : R * R);
            const float lo_k = bk > 0 ? bin_edge(base, shift, bk - 1) : -1.f;
            if ((shift != kShift0 || top != top0) && bo >= bk0) {
                edge_o = edge_k;
                upto_o = upto_k;
            }
            edge_o = fminf(edge_o, edge_k);

            const bool listed = gn <= kWqGather;
            // the list: the count scan's (gd, gs), or the gather scan's, in
            // the same space (Ld = gd, Ls after capq entries)
            float *Ld = gd;
            uint32_t *Ls = listed ? gs : (uint32_t *)(wb + L::ls(capq));
            int cnt = 0;
            if (listed) {
                // ------------- the count scan's list, cut to the Ndens-th bin
                for (int e0 = 0; e0 < gn; e0 += 32) {
                    const int e = e0 + lane;
                    float v = 0.f;
                    uint32_t sv = 0;
                    bool keep = false;
                    if (e < gn) {
                        v = gd[e];
                        sv = gs[e];
                        keep = v <= edge_k;
                    }
                    const uint32_t bal = __ballot_sync(kAll, keep);
                    const int pos = cnt + __popc(bal & lt);
                    __syncwarp();
                    if (keep) {
                        gd[pos] = v;
                        gs[pos] = sv;
                    }
                    cnt += __popc(bal);
                    __syncwarp();
                }
            } else {
            // ------------- scan B: gather every entry up to the Ndens-th bin,
            // from the cells that meet its ball
            if (!full) {
                const float e2 = edge_k * 1.00001f + box * box * 1e-12f;
                int keep_n = 0;
                for (int c0 = 0; c0 < nc; c0 += 32) {
                    const int j = c0 + lane;
                    uint32_t ra = 0, ln = 0;
                    bool keep = false;
                    if (j < nc) {
                        ra = cra[j];
                        ln = cln[j];
                        keep = cmd[j] <= e2;
                    }
                    const uint32_t bal = __ballot_sync(kAll, keep);
                    __syncwarp();
                    const int pos = keep_n + __popc(bal & lt);
                    if (keep) {
                        cra[pos] = ra;
                        cln[pos] = ln;
                    }
                    keep_n += __popc(bal);
                    __syncwarp();
                }
                nc = keep_n;
                total = wq_prefix(cln, cpre, nc, lane);
            }
            {
                cand_acc += total;
                wq_visit(a.spos, cra, cpre, nc, total, lane, [&](const float4 &v, uint32_t s, bool valid) {
                    float d2 = INFINITY;
                    if (valid) {
                        float dx, dy, dz;
                        if (full) {
                            dx = wrapdiff(v.x, rqx, box, half);
                            dy = wrapdiff(v.y, rqy, box, half);
                            dz = wrapdiff(v.z, rqz, box, half);
                        } else if (shifted) {
                            dx = (fx && v.x >= half ? v.x - box : v.x) - qx;
                            dy = (fy && v.y >= half ? v.y - box : v.y) - qy;
                            dz = (fz && v.z >= half ? v.z - box : v.z) - qz;
                        } else {
                            dx = v.x - qx;
                            dy = v.y - qy;
                            dz = v.z - qz;
                        }
                        d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    }
                    const bool keep = valid && d2 <= edge_k;
                    const uint32_t bal = __ballot_sync(kAll, keep);
                    const int pos = cnt + __popc(bal & lt);
                    if (keep && pos < capq) {
                        Ld[pos] = d2;
                        Ls[pos] = s;
                    }
                    cnt += __popc(bal);
                });
            }
            }
            __syncwarp();
            if (cnt != upto_k) {
                // the two scans disagree: cannot happen with exact arithmetic
                if (lane == 0) atomicOr(a.err, kErrKnnRetry);
                continue;
            }
            // ------------- selection (the list is in Ld / Ls)
            const float vk = wq_list_kth(Ld, cnt, lo_k, below_k, upto_k, k, kd, lane, lt);
            unsigned long long wsum = 0;
            const float rk = sqrtf(vk);
            const float inv_h = vk > 0.f ? 2.f / rk : 0.f;
            for (int e = lane; e < cnt; e += 32) {
                const float v = Ld[e];
                if (v < vk) {
                    const float w = m4<float>(sqrtf(v) * inv_h);
                    wsum += (unsigned long long)(w * 4294967296.0f + 0.5f);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(kAll, wsum, o);
            if (n_out > 0) {
                if (upto_o <= 32) {
                    // at most 32 entries up to the n_out-th bin: one per lane,
                    // sorted across the warp by (d^2, original index)
                    int no = 0;
                    for (int e0 = 0; e0 < cnt; e0 += 32) {
                        const int e = e0 + lane;
                        const float v = e < cnt ? Ld[e] : 0.f;
                        const bool in = e < cnt && v <= edge_o;
                        const uint32_t bal = __ballot_sync(kAll, in);
                        const int pos = no + __popc(bal & lt);
                        if (in && pos < 32) {
                            od[pos] = v;
                            os[pos] = Ls[e];
                        }
                        no += __popc(bal);
                    }
                    __syncwarp();
                    // sorted by d^2 first (a float key); equal distances, if
                    // any, are sorted again by (d^2, original index)
                    float fk = INFINITY;
                    uint32_t pay = 0u;
                    if (lane < no) {
                        pay = os[lane];
                        fk = od[lane];
                    }
                    warp_sort32_kv(fk, pay, lane);
                    const float prev = __shfl_up_sync(kAll, fk, 1);
                    if (__any_sync(kAll, lane > 0 && lane < no && prev == fk)) {
                        unsigned long long key = ~0ull;
                        if (lane < no) key = ((unsigned long long)__float_as_uint(fk) << 32) | __float_as_uint(a.spos[pay].w);
                        pay = wq_tie_sort(key, pay, lane);
                    }
                    if (lane < min(no, n_out)) a.nbr_s[(size_t)sq * a.ld_out + lane] = pay;
                } else {
                    wq_rank_in_list(Ld, Ls, cnt, edge_o, n_out, a.spos, a.nbr_s + (size_t)sq * a.ld_out, lane);
                }
            }
            if (lane == 0) {
                float dens;
                if (vk > 0.f) {
                    const float h = rk * 0.5f;
                    dens = (float)(norm * ((float)wsum * 2.3283064365386963e-10f) / (h * h * h));
                } else {
                    dens = INFINITY;
                }
                a.dens_s[sq] = dens;
                if (a.rk_s) a.rk_s[sq] = rk;
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        atomicAdd(&a.counters[kCntCand], cand_acc);
        atomicAdd(&a.counters[kCntSearch], (unsigned long long)search_acc);
        atomicAdd(&a.counters[kCntRetry], (unsigned long long)retry_acc);
        atomicAdd(&a.counters[kCntWarps], (unsigned long long)warp_acc);
    }
}

template <bool SEG> int knn_wq_run(hop_ctx *c, const KnnArgs &ka, int cpr)
{
    CgDev d;
    d.spos = (const float4 *)ka.spos;
    d.keys = ka.keys;
    d.cellT = ka.cellT;
    d.level_dense = ka.level_dense;
    d.n = ka.n;
    d.n_chunks = SEG ? ka.n_chunks : (ka.n + kWqChunk - 1) / kWqChunk;
    d.box = (float)ka.box;
    d.inv_box = (float)(1.0 / ka.box);
    d.half_box = (float)(0.5 * ka.box);
    d.norm = (float)(ka.box * ka.box * ka.box / ((double)(ka.n_norm > 0 ? ka.n_norm : ka.n) * 3.14159265358979323846));
    d.k = ka.k;
    d.n_out = ka.n_out;
    d.ld_out = ka.ld_out;
    d.capq = ((ka.k + 32 + 7) / 8) * 8;
    d.chunk_r = ka.chunk_r;
    d.plain_r = ka.plain_r;
    d.cpr = cpr;
    d.seg = ka.seg;
    d.B = ka.B;
    d.nbr_s = ka.nbr_s;
    d.dens_s = ka.dens_s;
    d.rk_s = ka.rk_s;
    d.counters = c->d_counters;
    d.chunk_counter = c->d_counters + kCntNum;
    d.err = c->d_err;
    HOP_CUDA(c, cudaMemsetAsync(d.chunk_counter, 0, sizeof(unsigned long long), c->stream));
    const size_t per_warp = WqSmem::total(d.capq);
    const int warps = kCgWarps;
    const size_t smem = per_warp * warps;
    auto kern = knn_wq_kernel<SEG>;
    HOP_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    HOP_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
    if (per_sm < 1) return ctx_fail(c, HOP_EINVAL, "kNN list does not fit in shared memory");
    int64_t blocks = (int64_t)per_sm * c->num_sms;
    const int64_t need = (d.n_chunks + warps - 1) / warps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, warps * 32, smem, c->stream>>>(d);
    HOP_LAUNCH(c);
    return HOP_OK;
}

template <int P, bool SEG> int knn_cg_run(hop_ctx *c, const KnnArgs &ka, int cpr)
{
    constexpr int Q = 32 / P;
    CgDev d;
    d.spos = (const float4 *)ka.spos;
    d.keys = ka.keys;
    d.cellT = ka.cellT;
    d.level_dense = ka.level_dense;
    d.n = ka.n;
    d.n_chunks = SEG ? ka.n_chunks : (ka.n + Q - 1) / Q;
    d.box = (float)ka.box;
    d.inv_box = (float)(1.0 / ka.box);
    d.half_box = (float)(0.5 * ka.box);
    d.norm = (float)(ka.box * ka.box * ka.box / ((double)(ka.n_norm > 0 ? ka.n_norm : ka.n) * 3.14159265358979323846));
    d.k = ka.k;
    d.n_out = ka.n_out;
    d.ld_out = ka.ld_out;
    // list room per query: Ndens plus the entries of the Ndens-th bin (a
    // quarter octave of d^2 holds about a sixth of Ndens); a crowded bin is
    // refined until the list fits
    d.capq = ((ka.k + 32 + 7) / 8) * 8;
    d.chunk_r = ka.chunk_r;
    d.plain_r = ka.plain_r;
    d.cpr = cpr;
    d.seg = ka.seg;
    d.B = ka.B;
    d.nbr_s = ka.nbr_s;
    d.dens_s = ka.dens_s;
    d.rk_s = ka.rk_s;
    d.counters = c->d_counters;
    d.chunk_counter = c->d_counters + kCntNum;
    d.err = c->d_err;
    HOP_CUDA(c, cudaMemsetAsync(d.chunk_counter, 0, sizeof(unsigned long long), c->stream));
    const size_t per_warp = CgSmem<Q>::total(d.capq);
    int max_smem = 0;
    HOP_CUDA(c, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    int warps = kCgWarps;
    while (warps > 1 && per_warp * warps > (size_t)max_smem) warps >>= 1;
    if (per_warp * warps > (size_t)max_smem)
        return ctx_fail(c, HOP_EINVAL, "kNN list does not fit in shared memory");
    const size_t smem = per_warp * warps;
    auto kern = knn_cg_kernel<P, SEG>;
    HOP_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    HOP_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
    if (per_sm < 1) return ctx_fail(c, HOP_EINVAL, "kNN list does not fit in shared memory");
    int64_t blocks = (int64_t)per_sm * c->num_sms;
    const int64_t need = (d.n_chunks + warps - 1) / warps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, warps * 32, smem, c->stream>>>(d);
    HOP_LAUNCH(c);
    return HOP_OK;
}

}  // namespace

int knn_cg_launch(hop_ctx *c, const KnnArgs &a, int qpw, int cpr)
{
    switch (qpw) {
    case 16: return a.seg ? knn_cg_run<2, true>(c, a, cpr) : knn_cg_run<2, false>(c, a, cpr);
    case 8: return a.seg ? knn_cg_run<4, true>(c, a, cpr) : knn_cg_run<4, false>(c, a, cpr);
    case 4: return a.seg ? knn_wq_run<true>(c, a, cpr) : knn_wq_run<false>(c, a, cpr);
    default: return ctx_fail(c, HOP_EINVAL, "count-then-gather kNN takes 4, 8 or 16 queries per warp");
    }
}
