// Certified kNN + M4 density with one query per lane (HOP step 1, Parallel
// HOP Sec. 2): the kernel for 32 queries per warp, float32 positions.
//
// Work unit.  A warp takes a chunk of 32 consecutive sorted particles (one
// subvolume) and gives each lane one query.  Consecutive queries closer
// than R stay in one group; a group's search region is its queries'
// bounding box grown by R, so a chunk that straddles a jump of the Morton
// curve is searched as two (or more) compact regions instead of one large
// one.  For each group the warp walks the cells (side >= R / cpr) that meet
// the region, stages their particles in shared memory (each staged particle
// passes a box-distance test against the region) and then every lane reads
// every staged particle -- one broadcast shared-memory load per particle for
// all 32 queries -- and tests it against its own query.
//
// Selection.  A lane keeps every particle it has seen with d^2 <= tau in
// its own list (shared memory, entry e of lane l at e * 32 + l, so appends
// never conflict), tau starting at R^2.  When a list nears its capacity the
// warp compacts: each filling lane histograms its list in 1/8-octave bins
// of d^2 below its largest entry, and tau drops to the upper edge of the
// bin holding the Ndens-th entry (or, in a crowded bin, to the exact
// Ndens-th value), so tau stays an upper bound of the Ndens-th distance of
// the particles seen.  A lane is certified when its list holds >= Ndens
// entries after a search with radius R: every particle within R of its
// query was tested, so the Ndens nearest are in the list.  Lanes not
// certified repeat with a larger R; certified lanes keep their lists.
//
// Results equal those of the kernel with several lanes per query: the same
// per-component differences (the frame shift x >= L/2 -> x - L on axes
// whose region crosses a face is exact), the same fused d^2, the same exact
// k-th distance and (d^2, original index) order, the same fixed-point sum
// of kernel weights.
#include "hop_internal.cuh"
#include "knn_common.cuh"

#include <math.h>

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kTile = 128;             // staged candidates per tile
constexpr int kPer = kTile / 32;       // candidates each lane loads per tile
constexpr int kTries = 96;

struct Cand {
    float x, y, z;
    uint32_t s;
};

struct K32 {
    const float4 *spos;
    const uint64_t *keys;
    const uint32_t *cellT;
    int level_dense;
    int64_t n, n_chunks;
    float box, inv_box, half_box, norm;
    int k, n_out, ld_out, cap;
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

// Shared memory of one warp (one warp per block), byte offsets.
struct K32Smem {
    static constexpr size_t tile = 0;                                   // kTile candidates
    static constexpr size_t rs = tile + sizeof(Cand) * kTile;           // 32 range starts
    static constexpr size_t ro = rs + 32 * 4;                           // 33 prefix offsets
    static constexpr size_t hist = (ro + 33 * 4 + 15) & ~size_t(15);    // 32 bins x 32 lanes
    static constexpr size_t list = hist + 32 * 32 * 4;   // cap + 1 rows: the last takes rejected tests
    __host__ __device__ static size_t idl(int cap) { return list + (size_t)(cap + 1) * 32 * 4; }
    __host__ __device__ static size_t total(int cap) { return list + (size_t)(cap + 1) * 32 * 8; }
};

__device__ __forceinline__ float wmin(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float wmax(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ int wmax_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Distance from a point (or a box [a, b]) to the box [lo, hi] along one
// axis, made smaller by eps so that rounding never drops a needed cell or
// particle.
__device__ __forceinline__ float gap(float a, float b, float lo, float hi, float eps)
{
    return fmaxf(0.f, fmaxf(lo - b, a - hi) - eps);
}

// Histogram of each needing lane's list in 32 bins of 1/8 octave of d^2
// below tau (below its largest entry while tau is infinite); returns the bin
// of the k-th entry, the entries below that bin and up to it, and the window
// base.  While the k-th entry falls in the open lowest bin the window moves
// 30 bins down, so the old lowest bin is resolved by the new bins 0..30.
__device__ void lane_hist(bool need, const float *d2l, int cnt, int cmax, int *hist, int lane, int k,
                          float tau, int &tb, int &bk, int &below, int &upto)
{
    float vtop = tau;
    if (__any_sync(kFull, need && !(tau < INFINITY))) {
        vtop = 0.f;
        #pragma unroll 4
        for (int e = 0; e < cmax; ++e)
            if (need && e < cnt) vtop = fmaxf(vtop, d2l[e * 32 + lane]);
    }
    tb = bin_base(vtop);
    bk = kHistBins - 1;
    below = 0;
    upto = 0;
    bool redo = need;
    for (int it = 0; it < 8 && __any_sync(kFull, redo); ++it) {
        if (redo) {
#pragma unroll
            for (int b = 0; b < kHistBins; ++b) hist[b * 32 + lane] = 0;
        }
        #pragma unroll 4
        for (int e = 0; e < cmax; ++e)
            if (redo && e < cnt) atomicAdd(&hist[bin_of(d2l[e * 32 + lane], tb) * 32 + lane], 1);
        __syncwarp();
        if (redo) {
            bool found = false;
            int cum = 0;
#pragma unroll
            for (int b = 0; b < kHistBins; ++b) {
                const int h = hist[b * 32 + lane];
                if (!found && cum + h >= k) {
                    found = true;
                    bk = b;
                    below = cum;
                    upto = cum + h;
                }
                cum += h;
            }
            if (!found) {
                bk = kHistBins - 1;
                below = cum;
                upto = cum;
            }
            if (found && bk == 0 && tb > kHistBins && it < 7) tb -= kHistBins - 2;
            else redo = false;
        }
    }
}

// Radix descent inside the window bin bk (0 < bk; its entries share the
// top 12 bits of their float pattern, d^2 >= 0 ordering like its bits):
// 5 bits per level, each level a 32-bin histogram of the entries that
// share the prefix so far, until the sub-bin holding the k-th entry holds
// at most stop_m entries, or the entries up to it number at most
// stop_upto, or it is a single value.  On return `below` counts the
// entries under the sub-bin, `upto` those up to it, and the sub-bin is the
// values whose bits >> shift equal pfx.
__device__ void lane_refine(bool need, const float *d2l, int cnt, int cmax, int *hist, int lane, int k,
                            int tb, int bk, int stop_m, int stop_upto, int &below, int &upto, uint32_t &pfx,
                            int &shift)
{
    pfx = (uint32_t)(tb - (kHistBins - 1) + bk);
    shift = 20;
    bool go = need && bk > 0 && upto - below > stop_m && upto > stop_upto;
    while (__any_sync(kFull, go)) {
        const int sh = shift - 5;
        if (go) {
#pragma unroll
            for (int b = 0; b < kHistBins; ++b) hist[b * 32 + lane] = 0;
        }
        #pragma unroll 4
        for (int e = 0; e < cmax; ++e) {
            if (go && e < cnt) {
                const uint32_t u = __float_as_uint(d2l[e * 32 + lane]);
                if ((u >> shift) == pfx) atomicAdd(&hist[((u >> sh) & 31u) * 32 + lane], 1);
            }
        }
        __syncwarp();
        if (go) {
            // first digit whose running count reaches k (the prefix holds the
            // k-th entry, so one does)
            int cum = below, d = 31, nb = below, nu = upto;
            bool found = false;
#pragma unroll
            for (int b = 0; b < kHistBins; ++b) {
                const int h = hist[b * 32 + lane];
                if (!found && cum + h >= k) {
                    found = true;
                    d = b;
                    nb = cum;
                    nu = cum + h;
                }
                cum += h;
            }
            below = nb;
            upto = nu;
            pfx = (pfx << 5) | (uint32_t)d;
            shift = sh;
            go = shift > 0 && upto - below > stop_m && upto > stop_upto;
        }
        __syncwarp();
    }
}

// Exact k-th smallest d^2 of a lane's list (window bin bk, `below` entries
// under it, `upto` up to it): radix descent until at most 32 candidates
// remain, which are gathered and ranked; a crowded open lowest bin (values
// next to zero) is ranked in place.
__device__ float lane_kth(bool need, const float *d2l, int cnt, int cmax, int *hist, int lane, int k,
                          int tb, int bk, int below, int upto)
{
    float *scr = (float *)hist;
    uint32_t pfx;
    int shift;
    const bool open = bk == 0;
    lane_refine(need && !open, d2l, cnt, cmax, hist, lane, k, tb, bk, 32, -1, below, upto, pfx, shift);
    const int m = upto - below;
    float vk = 0.f;
    const bool small = need && !open && m <= 32;
    const int mmax = wmax_i(small ? m : 0);
    if (mmax > 0) {
        int j = 0;
        #pragma unroll 4
        for (int e = 0; e < cmax; ++e) {
            if (small && e < cnt) {
                const float v = d2l[e * 32 + lane];
                if ((__float_as_uint(v) >> shift) == pfx) scr[(j++) * 32 + lane] = v;
            }
        }
        #pragma unroll 4
        for (int a = 0; a < mmax; ++a) {
            const bool mine = small && a < m;
            const float v = mine ? scr[a * 32 + lane] : 0.f;
            int lt = below, le = below;
            #pragma unroll 4
            for (int f = 0; f < mmax; ++f) {
                if (f < m) {
                    const float u = scr[f * 32 + lane];
                    lt += u < v;
                    le += u <= v;
                }
            }
            if (mine && lt < k && k <= le) vk = v;
        }
    }
    const bool crowded = need && !small;
    if (__any_sync(kFull, crowded)) {
        #pragma unroll 4
        for (int e = 0; e < cmax; ++e) {
            if (!(crowded && e < cnt)) continue;
            const float v = d2l[e * 32 + lane];
            if (open ? bin_of(v, tb) != 0 : (__float_as_uint(v) >> shift) != pfx) continue;
            // rank in the whole list
            int lt = 0, le = 0;
            #pragma unroll 4
            for (int f = 0; f < cnt; ++f) {
                const float u = d2l[f * 32 + lane];
                lt += u < v;
                le += u <= v;
            }
            if (lt < k && k <= le) vk = v;
        }
    }
    __syncwarp();
    return vk;
}

// Shrinks the lists of the lanes holding >= k entries (see Selection
// above): tau drops to the upper edge of the smallest histogram or radix
// sub-bin that holds the k-th entry and leaves room in the list.
__device__ void lane_compact(bool need, float *d2l, uint32_t *idl, int &cnt, float &tau, int cap, int *hist,
                             int lane, int k, uint32_t *err)
{
    const int cmax = wmax_i(need ? cnt : 0);
    int tb, bk, below, upto;
    lane_hist(need, d2l, cnt, cmax, hist, lane, k, tau, tb, bk, below, upto);
    float ntau = -1.f;
    if (need && bk > 0 && bk < kHistBins - 1 && upto <= cap - 16) ntau = bin_upper(0.f, tb, bk);
    // a crowded bin of a nearly full list: descend into it
    const bool deep = need && !(ntau >= 0.f) && cnt > cap - 16 && bk > 0;
    uint32_t pfx;
    int shift;
    lane_refine(deep, d2l, cnt, cmax, hist, lane, k, tb, bk, -1, cap - 16, below, upto, pfx, shift);
    if (deep) ntau = __uint_as_float(((pfx + 1u) << shift) - 1u);
    // the open lowest bin (d^2 next to zero): the exact k-th value
    const bool exact = need && !(ntau >= 0.f) && cnt > cap - 16;
    if (__any_sync(kFull, exact)) {
        const float vk = lane_kth(exact, d2l, cnt, cmax, hist, lane, k, tb, bk, below, upto);
        if (exact) ntau = vk;
    }
    if (need && ntau >= 0.f) {
        int j = 0;
        #pragma unroll 4
        for (int e = 0; e < cnt; ++e) {
            const float v = d2l[e * 32 + lane];
            if (v <= ntau) {
                d2l[j * 32 + lane] = v;
                idl[j * 32 + lane] = idl[e * 32 + lane];
                ++j;
            }
        }
        cnt = j;
        tau = fminf(tau, ntau);
    }
    if (need && cnt > cap - 8) {
        atomicOr(err, kErrDegenerate);
        cnt = cap - 8;
    }
    __syncwarp();
}

template <bool SEG>
__global__ void __launch_bounds__(32) knn32_kernel(K32 a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x;
    const uint32_t lt_mask = (1u << lane) - 1u;
    Cand *tile = (Cand *)(smem_raw + K32Smem::tile);
    uint32_t *rs = (uint32_t *)(smem_raw + K32Smem::rs);
    uint32_t *ro = (uint32_t *)(smem_raw + K32Smem::ro);
    int *hist = (int *)(smem_raw + K32Smem::hist);
    float *d2l = (float *)(smem_raw + K32Smem::list);
    uint32_t *idl = (uint32_t *)(smem_raw + K32Smem::idl(a.cap));
    const int k = a.k, cap = a.cap;
    unsigned long long cand_acc = 0, search_acc = 0, retry_acc = 0, warp_acc = 0;

    for (;;) {
        unsigned long long ch = 0;
        if (lane == 0) ch = atomicAdd(a.chunk_counter, 1ull);
        ch = __shfl_sync(kFull, ch, 0);
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
            s_first = sd.base + ((int64_t)ch - sd.chunk0) * 32;
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
            s_first = (int64_t)ch * 32;
            box = a.box;
            half = a.half_box;
            inv_box = a.inv_box;
            norm = a.norm;
            cellT = a.cellT;
            level_dense = a.level_dense;
            plain_r = a.plain_r;
        }
        const int nq = (int)min((int64_t)32, n_end - s_first);
        const bool active = lane < nq;
        const int64_t sq = s_first + (active ? lane : 0);
        const float4 qv = a.spos[sq];
        const float rqx = qv.x, rqy = qv.y, rqz = qv.z;
        const float eps = box * 9.5367431640625e-7f;   // 2^-20 of the box: far above coordinate rounding

        float R = a.chunk_r ? a.chunk_r[ch] : plain_r;
        if (!(R > 0.f)) R = box * 1e-6f;
        int cnt = 0;
        float tau = -1.f;
        bool done = !active;
        bool failed = false;
        int tries = 0;

        for (;;) {
            ++search_acc;
            const bool full = 2.f * R >= half;
            const bool want = !done;
            if (want) {
                cnt = 0;
                tau = full ? INFINITY : R * R;
            }
            const float R2c = R * R * 1.00001f + box * box * 1e-12f;
            // groups of consecutive queries (a cut where a query is more than R
            // from the one before it)
            const float px = __shfl_up_sync(kFull, rqx, 1), py = __shfl_up_sync(kFull, rqy, 1),
                        pz = __shfl_up_sync(kFull, rqz, 1);
            const float cx = rqx - px, cy = rqy - py, cz = rqz - pz;
            const bool cut = lane > 0 && !full && cx * cx + cy * cy + cz * cz > R * R;
            const uint32_t cuts = __ballot_sync(kFull, cut);
            const int gid = __popc(cuts & (lt_mask | (1u << lane)));
            const int ngroups = __popc(cuts) + 1;

            for (int g = 0; g < ngroups; ++g) {
                const bool member = want && gid == g;
                const uint32_t members = __ballot_sync(kFull, member);
                if (!members) continue;
                const int nmem = __popc(members);
                // frame of this group's region
                const float lx = wmin(member ? rqx : INFINITY), hx = wmax(member ? rqx : -INFINITY);
                const float ly = wmin(member ? rqy : INFINITY), hy = wmax(member ? rqy : -INFINITY);
                const float lz = wmin(member ? rqz : INFINITY), hz = wmax(member ? rqz : -INFINITY);
                const bool wx = lx - R < 0.f || hx + R >= box;
                const bool wy = ly - R < 0.f || hy + R >= box;
                const bool wz = lz - R < 0.f || hz + R >= box;
                const bool mixed = (wx && lx - R < half && half <= hx + R) ||
                                   (wy && ly - R < half && half <= hy + R) ||
                                   (wz && lz - R < half && half <= hz + R);
                const bool pairwrap = full || mixed;
                const float qx = (!pairwrap && wx && rqx >= half) ? rqx - box : rqx;
                const float qy = (!pairwrap && wy && rqy >= half) ? rqy - box : rqy;
                const float qz = (!pairwrap && wz && rqz >= half) ? rqz - box : rqz;
                const float flx = wmin(member ? qx : INFINITY), fhx = wmax(member ? qx : -INFINITY);
                const float fly = wmin(member ? qy : INFINITY), fhy = wmax(member ? qy : -INFINITY);
                const float flz = wmin(member ? qz : INFINITY), fhz = wmax(member ? qz : -INFINITY);

                int l = 1, G = 2;
                if (!full) {
                    const float cells = box * (float)a.cpr / R;   // 2^l <= cells: side >= R / cpr
                    while (l < kMaxLevel && (float)(1 << (l + 1)) <= cells) ++l;
                    G = 1 << l;
                }
                const float sc = inv_box * (float)G;
                const float csz = box / (float)G;
                int c0x = 0, c0y = 0, c0z = 0, nx = 1, ny = 1, nz = 1;
                if (!full) {
                    c0x = (int)floorf((flx - R) * sc);
                    c0y = (int)floorf((fly - R) * sc);
                    c0z = (int)floorf((flz - R) * sc);
                    nx = (int)floorf((fhx + R) * sc) - c0x + 1;
                    ny = (int)floorf((fhy + R) * sc) - c0y + 1;
                    nz = (int)floorf((fhz + R) * sc) - c0z + 1;
                    if (nx >= G) { c0x = 0; nx = G; }
                    if (ny >= G) { c0y = 0; ny = G; }
                    if (nz >= G) { c0z = 0; nz = G; }
                }
                const int ncells = nx * ny * nz;
                // two sweeps: the cells that meet the queries' box, then the
                // rest of the region; after the first, lanes holding Ndens
                // entries cut tau to their Ndens-th bin, so the outer cells
                // add few entries
                const int nsweeps = (full || pairwrap) ? 1 : 2;
                for (int sweep = 0; sweep < nsweeps; ++sweep) {
                if (sweep == 1 && __any_sync(kFull, member && cnt >= k))
                    lane_compact(member && cnt >= k, d2l, idl, cnt, tau, cap, hist, lane, k, a.err);
                for (int cb = 0; cb < ncells; cb += 32) {
                    // ---- ranges of up to 32 cells and their prefix
                    uint32_t ra = 0, rb = 0;
                    const int ci = cb + lane;
                    if (full) {
                        if (lane == 0) { ra = (uint32_t)seg_base; rb = (uint32_t)n_end; }
                    } else if (ci < ncells) {
                        const int ix = c0x + ci % nx, iy = c0y + (ci / nx) % ny, iz = c0z + ci / (nx * ny);
                        bool keep = true;
                        if (!pairwrap) {
                            // cell box (frame coordinates) against the region
                            const float gx = gap(ix * csz, (ix + 1) * csz, flx, fhx, eps);
                            const float gy = gap(iy * csz, (iy + 1) * csz, fly, fhy, eps);
                            const float gz = gap(iz * csz, (iz + 1) * csz, flz, fhz, eps);
                            const float g2 = gx * gx + gy * gy + gz * gz;
                            keep = sweep == 0 ? g2 == 0.f : (g2 > 0.f && g2 <= R2c);
                        }
                        if (keep) {
                            const int rx = ((ix % G) + G) % G, ry = ((iy % G) + G) % G, rz = ((iz % G) + G) % G;
                            cell_range(cellT, a.keys, level_dense, l,
                                       morton3((uint32_t)rx, (uint32_t)ry, (uint32_t)rz), ra, rb);
                        }
                    }
                    const uint32_t len = rb - ra;
                    uint32_t inc = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(kFull, inc, o);
                        if (lane >= o) inc += y;
                    }
                    const uint32_t total = __shfl_sync(kFull, inc, 31);
                    __syncwarp();
                    rs[lane] = ra;
                    ro[lane] = inc - len;
                    if (lane == 31) ro[32] = inc;
                    __syncwarp();

                    // ---- stream the candidates through the tile; the next
                    // tile's loads are issued before the current one is tested
                    float4 pv[kPer];
                    uint32_t pidx[kPer];
                    int cur = 0;
                    auto fetch = [&](uint32_t t0) {
#pragma unroll
                        for (int jj = 0; jj < kPer; ++jj) {
                            const uint32_t gi = t0 + (uint32_t)(lane + 32 * jj);
                            pidx[jj] = 0xffffffffu;
                            if (gi < total) {
                                while (ro[cur + 1] <= gi) ++cur;
                                pidx[jj] = rs[cur] + (gi - ro[cur]);
                            }
                        }
#pragma unroll
                        for (int jj = 0; jj < kPer; ++jj)
                            if (pidx[jj] != 0xffffffffu) pv[jj] = a.spos[pidx[jj]];
                    };
                    if (total > 0) fetch(0);
                    for (uint32_t t0 = 0; t0 < total; t0 += kTile) {
                        int m = 0;
#pragma unroll
                        for (int jj = 0; jj < kPer; ++jj) {
                            Cand c;
                            bool keep = false;
                            if (pidx[jj] != 0xffffffffu) {
                                const float4 v = pv[jj];
                                if (pairwrap) {
                                    c.x = v.x; c.y = v.y; c.z = v.z;
                                    keep = true;
                                } else {
                                    c.x = (wx && v.x >= half) ? v.x - box : v.x;
                                    c.y = (wy && v.y >= half) ? v.y - box : v.y;
                                    c.z = (wz && v.z >= half) ? v.z - box : v.z;
                                    const float gx = gap(c.x, c.x, flx, fhx, eps);
                                    const float gy = gap(c.y, c.y, fly, fhy, eps);
                                    const float gz = gap(c.z, c.z, flz, fhz, eps);
                                    keep = gx * gx + gy * gy + gz * gz <= R2c;
                                }
                                c.s = pidx[jj];
                            }
                            const uint32_t kb = __ballot_sync(kFull, keep);
                            if (keep) tile[m + __popc(kb & lt_mask)] = c;
                            m += __popc(kb);
                        }
                        // pad to a multiple of 8 with entries no test accepts
                        if (lane < ((8 - (m & 7)) & 7)) {
                            Cand z;
                            z.x = z.y = z.z = __int_as_float(0x7fc00000);
                            z.s = 0;
                            tile[m + lane] = z;
                        }
                        __syncwarp();
                        if (t0 + kTile < total) fetch(t0 + kTile);
                        cand_acc += (unsigned long long)m * (unsigned long long)nmem;
                        // ---- every lane tests every staged candidate
                        for (int j0 = 0; j0 < m; j0 += 8) {
                            float d2[8];
                            uint32_t sj[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const Cand c = tile[j0 + u];
                                float dx, dy, dz;
                                if (pairwrap) {
                                    dx = wrapdiff(c.x, rqx, box, half);
                                    dy = wrapdiff(c.y, rqy, box, half);
                                    dz = wrapdiff(c.z, rqz, box, half);
                                } else {
                                    dx = c.x - qx;
                                    dy = c.y - qy;
                                    dz = c.z - qz;
                                }
                                d2[u] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                                sj[u] = c.s;
                            }
                            // branch-free appends: a rejected test writes the spare row
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const bool acc = member && d2[u] <= tau;
                                const int row = acc ? cnt : cap;
                                d2l[row * 32 + lane] = d2[u];
                                idl[row * 32 + lane] = sj[u];
                                cnt += acc ? 1 : 0;
                            }
                            if (__any_sync(kFull, cnt > cap - 8))
                                lane_compact(cnt >= k, d2l, idl, cnt, tau, cap, hist, lane, k, a.err);
                        }
                        __syncwarp();
                    }
                }
                }
            }
            // ---- certification
            const bool ok = !want || cnt >= k;
            if (want && ok) done = true;
            if (__all_sync(kFull, done)) break;
            ++retry_acc;
            if (++tries >= kTries || full) {
                if (lane == 0) atomicOr(a.err, kErrKnnRetry);
                failed = true;
                break;
            }
            float f = 1.25f;
            if (!ok) f = fmaxf(f, 1.1f * cbrtf((float)k / (float)max(cnt, 1)));
            f = wmax(f);
            R *= fminf(f, 8.f);
        }
        if (failed) continue;

        // -------------------- selection (each lane its own query)
        {
            const bool need = active;
            const int n_out = (a.nbr_s != nullptr) ? a.n_out : 0;
            const int cmax = wmax_i(need ? cnt : 0);
            int tb, bk, below_k, upto_k;
            lane_hist(need, d2l, cnt, cmax, hist, lane, k, tau, tb, bk, below_k, upto_k);
            // bin of the n_out-th entry, from the same histogram
            int bo = 0, upto_o = 0;
            if (n_out > 0) {
                int cum = 0;
                bool found = false;
#pragma unroll
                for (int b = 0; b < kHistBins; ++b) {
                    const int h = hist[b * 32 + lane];
                    if (!found && cum + h >= n_out) {
                        found = true;
                        bo = b;
                        upto_o = cum + h;
                    }
                    cum += h;
                }
            }
            __syncwarp();
            const float vk = lane_kth(need, d2l, cnt, cmax, hist, lane, k, tb, bk, below_k, upto_k);
            // density: fixed-point sum of w(2 r / r_k) over entries with d^2 < r_k^2
            unsigned long long wsum = 0;
            const float rk = sqrtf(vk);
            const float inv_h = vk > 0.f ? 2.f / rk : 0.f;
            #pragma unroll 4
            for (int e = 0; e < cmax; ++e) {
                if (need && e < cnt) {
                    const float v = d2l[e * 32 + lane];
                    if (v < vk) {
                        const float w = m4<float>(sqrtf(v) * inv_h);
                        wsum += (unsigned long long)(w * 4294967296.0f + 0.5f);
                    }
                }
            }
            // the n_out nearest in (d^2, original index) order: the entries up
            // to the n_out-th entry's bin, gathered (24 per lane) and ranked
            if (n_out > 0) {
                // scratch: tile, ranges and histogram are free now (6 KB)
                float *sd = (float *)smem_raw;                          // 24 x 32 d^2 ...
                uint32_t *si = (uint32_t *)(smem_raw + 24 * 32 * 4);    // ... and sorted indices
                static_assert(24 * 32 * 8 <= K32Smem::list, "selection scratch");
                const bool small = upto_o <= 24;
                const int momax = wmax_i((need && small) ? upto_o : 0);
                __syncwarp();
                if (momax > 0) {
                    int j = 0;
                    #pragma unroll 4
                    for (int e = 0; e < cmax; ++e) {
                        if (need && small && e < cnt) {
                            const float v = d2l[e * 32 + lane];
                            if (bin_of(v, tb) <= bo) {
                                sd[j * 32 + lane] = v;
                                si[j * 32 + lane] = idl[e * 32 + lane];
                                ++j;
                            }
                        }
                    }
                    #pragma unroll 4
                    for (int e = 0; e < momax; ++e) {
                        const bool mine = need && small && e < upto_o;
                        const float v = mine ? sd[e * 32 + lane] : 0.f;
                        const uint32_t se = mine ? si[e * 32 + lane] : 0u;
                        uint32_t oe = 0xffffffffu;
                        int rank = 0;
                        #pragma unroll 4
                        for (int f = 0; f < momax; ++f) {
                            if (f < upto_o) {
                                const float u = sd[f * 32 + lane];
                                rank += u < v;
                                if (mine && u == v && f != e) {
                                    if (oe == 0xffffffffu) oe = __float_as_uint(a.spos[se].w);
                                    rank += __float_as_uint(a.spos[si[f * 32 + lane]].w) < oe;
                                }
                            }
                        }
                        if (mine && rank < n_out) a.nbr_s[(size_t)sq * a.ld_out + rank] = se;
                    }
                }
                if (__any_sync(kFull, need && !small)) {
                    #pragma unroll 4
                    for (int e = 0; e < cmax; ++e) {
                        if (!(need && !small && e < cnt)) continue;
                        const float v = d2l[e * 32 + lane];
                        if (bin_of(v, tb) > bo) continue;
                        const uint32_t se = idl[e * 32 + lane];
                        uint32_t oe = 0xffffffffu;
                        int rank = 0;
                        #pragma unroll 4
                        for (int f = 0; f < cnt; ++f) {
                            const float u = d2l[f * 32 + lane];
                            if (u < v) { ++rank; continue; }
                            if (u == v && f != e) {
                                if (oe == 0xffffffffu) oe = __float_as_uint(a.spos[se].w);
                                rank += __float_as_uint(a.spos[idl[f * 32 + lane]].w) < oe;
                            }
                        }
                        if (rank < n_out) a.nbr_s[(size_t)sq * a.ld_out + rank] = se;
                    }
                }
            }
            if (need) {
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
        }
        __syncwarp();
    }
    if (lane == 0) {
        atomicAdd(&a.counters[kCntCand], cand_acc);
        atomicAdd(&a.counters[kCntSearch], search_acc);
        atomicAdd(&a.counters[kCntRetry], retry_acc);
        atomicAdd(&a.counters[kCntWarps], warp_acc);
    }
}

template <bool SEG> int knn32_run(hop_ctx *c, const KnnArgs &ka, int cpr)
{
    K32 d;
    d.spos = (const float4 *)ka.spos;
    d.keys = ka.keys;
    d.cellT = ka.cellT;
    d.level_dense = ka.level_dense;
    d.n = ka.n;
    d.n_chunks = SEG ? ka.n_chunks : (ka.n + 31) / 32;
    d.box = (float)ka.box;
    d.inv_box = (float)(1.0 / ka.box);
    d.half_box = (float)(0.5 * ka.box);
    d.norm = (float)(ka.box * ka.box * ka.box / ((double)(ka.n_norm > 0 ? ka.n_norm : ka.n) * 3.14159265358979323846));
    d.k = ka.k;
    d.n_out = ka.n_out;
    d.ld_out = ka.ld_out;
    // list capacity per query: buffer factor x Ndens / 2 (default 2 Ndens),
    // at least Ndens + 32
    const int f = c->capf ? c->capf : 4;
    int cap = std::max(ka.k + 32, f * ka.k / 2);
    cap = (cap + 3) & ~3;
    d.cap = cap;
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
    const size_t smem = K32Smem::total(cap);
    int max_smem = 0;
    HOP_CUDA(c, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    if (smem > (size_t)max_smem) return ctx_fail(c, HOP_EINVAL, "kNN list does not fit in shared memory");
    auto kern = knn32_kernel<SEG>;
    HOP_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    HOP_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, smem));
    if (per_sm < 1) return ctx_fail(c, HOP_EINVAL, "kNN list does not fit in shared memory");
    int64_t blocks = (int64_t)per_sm * c->num_sms;
    if (blocks > d.n_chunks) blocks = d.n_chunks;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 32, smem, c->stream>>>(d);
    HOP_LAUNCH(c);
    return HOP_OK;
}

}  // namespace

int knn32_launch(hop_ctx *c, const KnnArgs &a, int cpr)
{
    return a.seg ? knn32_run<true>(c, a, cpr) : knn32_run<false>(c, a, cpr);
}
