// Certified cell-stencil kNN fused with the M4 cubic-spline density
// (HOP step 1, Parallel HOP Sec. 2).
//
// Layout.  Particles are sorted by a 48-bit Morton key, so every octree
// cell at every level 0..16 is one contiguous range of the sorted float4
// array {x, y, z, original index}.  A dense table gives the ranges of the
// cells at one level (about one particle per cell); deeper cells are found by
// binary search of the keys inside their dense ancestor.
//
// Work unit.  One warp takes Q = 32/P consecutive sorted particles (a chunk)
// and serves them with P lanes each.  For a search radius R the warp scans
// the cells (side >= R / cpr) lying within R of at least one of its queries;
// candidates are staged in shared memory (the next tile's loads are issued
// while the current tile is tested) and each lane tests every P-th staged
// candidate against its query.
//
// Selection.  A query keeps, in shared memory, every candidate seen so far
// with d^2 <= tau (tau starts at R^2).  When the buffer passes 4 Ndens the
// entries are histogrammed in 1/8-octave bins of d^2 below tau and tau drops
// to the upper edge of the bin holding the Ndens-th entry, so tau stays an
// upper bound of the Ndens-th distance of the candidates seen.  The search
// is certified when every query holds >= Ndens entries: then all particles
// within sqrt(tau) (<= R) were scanned and the Ndens nearest are exactly in
// the buffer.  Otherwise the warp repeats with a larger R.
//
// Distances.  Inside a warp the box is unwrapped on each axis whose search
// region crosses a face: coordinates >= L/2 move to x - L, exact by
// Sterbenz' lemma, so d^2 = (xj - xi)^2 + ... has one rounding per
// component difference whatever R was.  The density is a fixed-point sum of
// kernel weights, so results do not depend on R, on the radius policy or on
// the order candidates arrive in.
#include "hop_internal.cuh"
#include "knn_common.cuh"

#include <math.h>

namespace {

constexpr int kKnnWarps = 4;               // warps per block
constexpr int kKnnThreads = kKnnWarps * 32;
constexpr int kMaxTries = 96;
constexpr uint32_t FULL = 0xffffffffu;

template <typename T> struct Rec;
template <> struct Rec<float> { float x, y, z; uint32_t s; };
template <> struct Rec<double> { double x, y, z; uint32_t s; uint32_t pad; };

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4; };

template <typename T> __device__ __forceinline__ uint32_t orig_of(const typename V4<T>::type &v);
template <> __device__ __forceinline__ uint32_t orig_of<float>(const float4 &v) { return __float_as_uint(v.w); }
template <> __device__ __forceinline__ uint32_t orig_of<double>(const double4 &v)
{
    return (uint32_t)__double_as_longlong(v.w);
}

constexpr int KCAP = 32;   // entries of the k-th entry's bin ranked exactly in a small list
constexpr int OCAP = 64;   // candidates for the n_out nearest ranked in a small list

__device__ __forceinline__ int warp_max_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

template <typename T, int P> __device__ __forceinline__ T group_max(T v)
{
#pragma unroll
    for (int o = 1; o < P; o <<= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// The selection helpers below are called by all 32 lanes of the warp with
// warp-uniform loop bounds (the largest buffer in the warp); `need` masks
// the query groups they act for.  Every group then runs the same
// instruction stream instead of its own data-dependent loops one after the
// other.

// Histogram of each needing group's buffer in 1/8-octave bins of d^2 below
// its largest entry; when the k-th (or n_out-th) entry falls in the lowest,
// open-ended bin the window moves 31 bins down.  Returns bk / bo (bins of
// the k-th and n_out-th entries), the entries below bk and up to bk, and
// the window base tb.
template <typename T, int P>
__device__ void warp_hist(bool need, const T *bd, int cnt, int cmax, int *hist, int k, int n_out,
                          int p, uint32_t gmask, int &tb, int &bk, int &bo, int &below_k, int &upto_k)
{
    T vmax = T(0);
    for (int e0 = 0; e0 < cmax; e0 += P) {
        const int e = e0 + p;
        if (need && e < cnt) vmax = max(vmax, bd[e]);
    }
    vmax = group_max<T, P>(vmax);
    tb = bin_base(vmax);
    bk = bo = kHistBins - 1;
    below_k = 0;
    upto_k = cnt;
    bool pending = need;
    for (int guard = 0; guard < 96; ++guard) {
        if (pending)
            for (int b = p; b < kHistBins; b += P) hist[b] = 0;
        __syncwarp();
        for (int e0 = 0; e0 < cmax; e0 += P) {
            const int e = e0 + p;
            if (pending && e < cnt) atomicAdd(&hist[bin_of(bd[e], tb)], 1);
        }
        __syncwarp();
        {
            // the group's P lanes each sum kHistBins/P consecutive bins; a
            // prefix over the group finds the lanes holding the k-th and
            // n_out-th entries, which then scan their own bins
            constexpr int PER = kHistBins / P;
            int mine = 0;
#pragma unroll
            for (int i = 0; i < PER; ++i) mine += pending ? hist[p * PER + i] : 0;
            int incl = mine;
#pragma unroll
            for (int o = 1; o < P; o <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, o, P);
                if (p >= o) incl += y;
            }
            const int excl = incl - mine;
            int fk = -1, fbelow = 0, fupto = 0, fo = -1;
            if (pending && excl < k && k <= incl) {
                int cum = excl;
                for (int i = 0; i < PER; ++i) {
                    const int h = hist[p * PER + i];
                    if (cum + h >= k) { fk = p * PER + i; fbelow = cum; fupto = cum + h; break; }
                    cum += h;
                }
            }
            if (pending && n_out > 0 && excl < n_out && n_out <= incl) {
                int cum = excl;
                for (int i = 0; i < PER; ++i) {
                    const int h = hist[p * PER + i];
                    if (cum + h >= n_out) { fo = p * PER + i; break; }
                    cum += h;
                }
            }
            const uint32_t hk = __ballot_sync(FULL, fk >= 0) & gmask;
            const uint32_t ho = __ballot_sync(FULL, fo >= 0) & gmask;
            const int lk = hk ? __ffs(hk) - 1 : 0, lo = ho ? __ffs(ho) - 1 : 0;
            const int gk = __shfl_sync(FULL, fk, lk), gbelow = __shfl_sync(FULL, fbelow, lk),
                      gupto = __shfl_sync(FULL, fupto, lk), go = __shfl_sync(FULL, fo, lo);
            if (pending) {
                bk = hk ? gk : kHistBins - 1;
                below_k = hk ? gbelow : 0;
                upto_k = hk ? gupto : cnt;
                bo = n_out <= 0 ? kHistBins - 1 : (ho ? go : kHistBins - 1);
            }
        }
        __syncwarp();
        const bool shift = pending && !((bk > 0 && bo > 0) || tb <= kHistBins);
        if (shift) tb -= kHistBins - 1;
        pending = shift;
        if (!__any_sync(FULL, pending)) break;
    }
}

// The same quantities as warp_hist, from the per-lane histogram rows kept
// up to date while appending (bins relative to the window base tbw): the
// group's P lanes each sum kHistBins/P bins over the P rows.  Returns false
// in `ok` when the k-th (or n_out-th) entry lies in the open-ended lowest bin,
// so the caller has to use warp_hist.
template <int P>
__device__ void rows_scan(bool need, const int *grows, int gtot, int k, int n_out, int p, uint32_t gmask,
                          int &bk, int &bo, int &below_k, int &upto_k, bool &ok)
{
    constexpr int PER = kHistBins / P;
    int mine = 0;
    if (need) {
#pragma unroll
        for (int r = 0; r < P; ++r)
#pragma unroll
            for (int i = 0; i < PER; ++i) mine += grows[r * (kHistBins + 1) + p * PER + i];
    }
    int incl = mine;
#pragma unroll
    for (int o = 1; o < P; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o, P);
        if (p >= o) incl += y;
    }
    const int excl = incl - mine;
    int fk = -1, fbelow = 0, fupto = 0, fo = -1;
    if (need && excl < k && k <= incl) {
        int cum = excl;
        for (int i = 0; i < PER; ++i) {
            int h = 0;
#pragma unroll
            for (int r = 0; r < P; ++r) h += grows[r * (kHistBins + 1) + p * PER + i];
            if (cum + h >= k) { fk = p * PER + i; fbelow = cum; fupto = cum + h; break; }
            cum += h;
        }
    }
    if (need && n_out > 0 && excl < n_out && n_out <= incl) {
        int cum = excl;
        for (int i = 0; i < PER; ++i) {
            int h = 0;
#pragma unroll
            for (int r = 0; r < P; ++r) h += grows[r * (kHistBins + 1) + p * PER + i];
            if (cum + h >= n_out) { fo = p * PER + i; break; }
            cum += h;
        }
    }
    const uint32_t hk = __ballot_sync(FULL, fk >= 0) & gmask;
    const uint32_t ho = __ballot_sync(FULL, fo >= 0) & gmask;
    const int lk = hk ? __ffs(hk) - 1 : 0, lo = ho ? __ffs(ho) - 1 : 0;
    const int gk = __shfl_sync(FULL, fk, lk), gbelow = __shfl_sync(FULL, fbelow, lk),
              gupto = __shfl_sync(FULL, fupto, lk), go = __shfl_sync(FULL, fo, lo);
    bk = hk ? gk : kHistBins - 1;
    below_k = hk ? gbelow : 0;
    upto_k = hk ? gupto : gtot;
    bo = n_out <= 0 ? kHistBins - 1 : (ho ? go : kHistBins - 1);
    ok = !need || (hk && bk > 0 && (n_out <= 0 || (ho && bo > 0)));
}

// Bit patterns of non-negative values, which order like the values; a
// window bin (0 < bin) holds the values sharing the top S0-shifted bits.
template <typename T> struct FBits;
template <> struct FBits<float> {
    using U = uint32_t;
    static constexpr int S0 = 20;
    __device__ static U of(float v) { return __float_as_uint(v); }
    __device__ static float val(U u) { return __uint_as_float(u); }
};
template <> struct FBits<double> {
    using U = unsigned long long;
    static constexpr int S0 = 49;
    __device__ static U of(double v) { return (U)__double_as_longlong(v); }
    __device__ static double val(U u) { return __longlong_as_double((long long)u); }
};

// Exact k-th smallest value of each needing group's buffer when its window
// bin bk (0 < bk; below entries under it, upto up to it) holds more than
// KCAP entries -- a dense clump at the k-th distance.  A radix descent on
// the bit pattern (5 bits per level, a 32-bin histogram of the bin's
// entries sharing the prefix so far, built by the group's P lanes) narrows
// the bin until at most KCAP entries, or a single value, remain; those are
// gathered and ranked.  A bin below the top shares the top bits of its
// values, so the descent starts there; the top bin also takes every value
// above the window (when the window was moved down), so there the descent
// starts from the full pattern.  Written to *out.
template <typename T, int P>
__device__ void warp_kth_deep(bool need, const T *bd, int cnt, int cmax, int *hist, int tb, int bk, int below,
                              int upto, int k, int p, uint32_t gmask, uint32_t lt_mask, T *kd, T *out)
{
    using B = FBits<T>;
    using U = typename B::U;
    constexpr int PER = kHistBins / P;
    constexpr int W = 8 * (int)sizeof(U);
    const bool top = bk == kHistBins - 1;
    U pfx = top ? U(0) : (U)(tb - (kHistBins - 1) + bk);
    int shift = top ? W : B::S0;
    // an entry of the sub-bin: in window bin bk and sharing the prefix
    auto match = [&](T v) {
        const U u = B::of(v);
        return (shift >= W || (u >> shift) == pfx) && (!top || bin_of(v, tb) == bk);
    };
    bool go = need && upto - below > KCAP;
    for (int guard = 0; guard < 16 && __any_sync(FULL, go); ++guard) {
        const int sh = shift > 5 ? shift - 5 : 0;
        const U dmask = (U(1) << (shift - sh)) - 1;
        if (go)
            for (int b = p; b < kHistBins; b += P) hist[b] = 0;
        __syncwarp();
        for (int e0 = 0; e0 < cmax; e0 += P) {
            const int e = e0 + p;
            if (go && e < cnt) {
                const T v = bd[e];
                if (match(v)) atomicAdd(&hist[(int)((B::of(v) >> sh) & dmask)], 1);
            }
        }
        __syncwarp();
        // the first digit whose running count reaches k: each lane sums
        // PER digits, a prefix over the group finds the lane that holds it
        int mine = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) mine += go ? hist[p * PER + i] : 0;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < P; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o, P);
            if (p >= o) incl += y;
        }
        const int excl = incl - mine;
        int fd = -1, fb = 0, fu = 0;
        if (go && below + excl < k && k <= below + incl) {
            int cum = below + excl;
            for (int i = 0; i < PER; ++i) {
                const int h = hist[p * PER + i];
                if (cum + h >= k) { fd = p * PER + i; fb = cum; fu = cum + h; break; }
                cum += h;
            }
        }
        const uint32_t hd = __ballot_sync(FULL, fd >= 0) & gmask;
        const int ld = hd ? __ffs(hd) - 1 : 0;
        const int gd = __shfl_sync(FULL, fd, ld), gb = __shfl_sync(FULL, fb, ld), gu = __shfl_sync(FULL, fu, ld);
        if (go) {
            if (hd) {
                pfx = shift >= W ? (U)gd : ((pfx << (shift - sh)) | (U)gd);
                below = gb;
                upto = gu;
                shift = sh;
            }
            go = hd && shift > 0 && upto - below > KCAP;
        }
        __syncwarp();
    }
    int nk = 0;
    for (int e0 = 0; e0 < cmax; e0 += P) {
        const int e = e0 + p;
        T v = T(0);
        bool in = false;
        if (need && e < cnt) {
            v = bd[e];
            in = match(v);
        }
        const uint32_t m = __ballot_sync(FULL, in) & gmask;
        if (in) {
            const int pos = nk + __popc(m & lt_mask);
            if (pos < KCAP) kd[pos] = v;
        }
        nk += __popc(m);
    }
    __syncwarp();
    const bool small = nk <= KCAP;
    // more than KCAP entries with the whole bit pattern in common: one value
    if (need && !small && p == 0) *out = B::val(shift >= W ? U(0) : (pfx << shift));
    const int nkmax = warp_max_i((need && small) ? nk : 0);
    for (int e0 = 0; e0 < nkmax; e0 += P) {
        const int e = e0 + p;
        const bool mine = need && small && e < nk;
        const T v = mine ? kd[e] : T(0);
        int lt = below, le = below;
        for (int f = 0; f < nkmax; ++f) {
            if (f < nk) {
                const T u = kd[f];
                lt += u < v;
                le += u <= v;
            }
        }
        if (mine && lt < k && k <= le) *out = v;
    }
    __syncwarp();
}

// Exact k-th smallest value of each needing group's buffer, given that it
// lies in bin bk with below_k smaller entries: the entries of bin bk are
// gathered into a small list and ranked there; a crowded bin goes through
// warp_kth_deep (the open lowest bin, values next to zero, is ranked in the
// whole buffer).  Written to *out.
template <typename T, int P>
__device__ void warp_kth(bool need, const T *bd, int cnt, int cmax, int *hist, int tb, int bk, int below_k,
                         int upto_k, int k, int p, uint32_t gmask, uint32_t lt_mask, T *kd, T *out)
{
    int nk = 0;
    for (int e0 = 0; e0 < cmax; e0 += P) {
        const int e = e0 + p;
        T v = T(0);
        bool in = false;
        if (need && e < cnt) {
            v = bd[e];
            in = bin_of(v, tb) == bk;
        }
        const uint32_t m = __ballot_sync(FULL, in) & gmask;
        if (in) {
            const int pos = nk + __popc(m & lt_mask);
            if (pos < KCAP) kd[pos] = v;
        }
        nk += __popc(m);
    }
    __syncwarp();
    const bool small = nk <= KCAP;
    const int nkmax = warp_max_i((need && small) ? nk : 0);
    for (int e0 = 0; e0 < nkmax; e0 += P) {
        const int e = e0 + p;
        const bool mine = need && small && e < nk;
        const T v = mine ? kd[e] : T(0);
        int lt = below_k, le = below_k;
        for (int f = 0; f < nkmax; ++f) {
            if (f < nk) {
                const T u = kd[f];
                lt += u < v;
                le += u <= v;
            }
        }
        if (mine && lt < k && k <= le) *out = v;
    }
    if (__any_sync(FULL, need && !small && bk > 0))
        warp_kth_deep<T, P>(need && !small && bk > 0, bd, cnt, cmax, hist, tb, bk, below_k, upto_k, k, p, gmask,
                            lt_mask, kd, out);
    if (__any_sync(FULL, need && !small && bk == 0)) {
        for (int e0 = 0; e0 < cmax; e0 += P) {
            const int e = e0 + p;
            if (need && !small && bk == 0 && e < cnt) {
                const T v = bd[e];
                if (bin_of(v, tb) == bk) {
                    int lt = below_k, le = below_k;
                    for (int f = 0; f < cnt; ++f) {
                        const T u = bd[f];
                        if (bin_of(u, tb) != bk) continue;
                        lt += u < v;
                        le += u <= v;
                    }
                    if (lt < k && k <= le) *out = v;
                }
            }
        }
    }
    __syncwarp();
}

// Keeps each needing group's entries with d^2 <= ntau, in order, in place
// (P entries per round: every read of a round precedes its writes).
template <typename T, int P>
__device__ void warp_compact(bool need, T *bd, uint32_t *bs, int &cnt, int cmax, T ntau, int p,
                             uint32_t gmask, uint32_t lt_mask)
{
    int wp = 0;
    for (int base = 0; base < cmax; base += P) {
        const int e = base + p;
        T v = T(0);
        uint32_t sv = 0;
        bool keep = false;
        if (need && e < cnt) {
            v = bd[e];
            sv = bs[e];
            keep = v <= ntau;
        }
        const uint32_t kb = __ballot_sync(FULL, keep) & gmask;
        __syncwarp();
        if (keep) {
            const int dst = wp + __popc(kb & lt_mask);
            bd[dst] = v;
            bs[dst] = sv;
        }
        wp += __popc(kb);
        __syncwarp();
    }
    if (need) cnt = wp;
}

template <typename T> struct KnnDev {
    const typename V4<T>::type *spos;
    const uint64_t *keys;
    const uint32_t *cellT;
    int level_dense;
    int64_t n;
    int64_t n_chunks;
    T box, inv_box, half_box;
    int k, n_out, ld_out, cap, buf;
    const float *chunk_r;
    float plain_r;
    int cpr;
    T norm;                       // box^3 / (n pi)
    const SegDesc *seg;           // subvolumes of a batched pass (SEG kernels)
    int B;
    uint32_t *nbr_s;
    float *dens_s;
    float *rk_s;
    unsigned long long *chunk_counter;
    unsigned long long *counters;
    uint32_t *err;
};

// Shared-memory layout of one warp (byte offsets), used by kernel and host.
template <typename T, int P> struct WarpSmem {
    static constexpr int Q = 32 / P;
    static constexpr int TILE = sizeof(T) == 4 ? 128 : 64;
    __host__ __device__ static size_t tile() { return 0; }
    __host__ __device__ static size_t bd() { return sizeof(Rec<T>) * TILE; }
    __host__ __device__ static size_t bs(int buf) { return bd() + sizeof(T) * (size_t)Q * buf; }
    __host__ __device__ static size_t hist(int buf) { return bs(buf) + sizeof(uint32_t) * (size_t)Q * buf; }
    __host__ __device__ static size_t rs(int buf) { return hist(buf) + sizeof(int) * Q * kHistBins; }
    __host__ __device__ static size_t kth(int buf) { return rs(buf) + 68 * 4; }        // rs[32], ro[33], pad
    __host__ __device__ static size_t qpos(int buf) { return kth(buf) + sizeof(T) * Q; }
    __host__ __device__ static size_t cube(int buf) { return qpos(buf) + sizeof(T) * 3 * Q; }
    __host__ __device__ static size_t hrow(int buf) { return (cube(buf) + sizeof(int) * 6 * Q + 15) & ~size_t(15); }
    __host__ __device__ static size_t kd(int buf) { return hrow(buf) + sizeof(int) * 32 * (kHistBins + 1); }
    __host__ __device__ static size_t od(int buf) { return kd(buf) + sizeof(T) * Q * KCAP; }
    __host__ __device__ static size_t os(int buf) { return od(buf) + sizeof(T) * Q * OCAP; }
    __host__ __device__ static size_t total(int buf)
    {
        return (os(buf) + sizeof(uint32_t) * Q * OCAP + 15) & ~size_t(15);
    }
};

// Is real cell (rx, ry, rz) inside the (periodic) cube c = {lo x3, n x3}?
__device__ __forceinline__ bool in_cube(const int *c, int rx, int ry, int rz, int G)
{
    return (((rx - c[0]) % G + G) % G) < c[3] && (((ry - c[1]) % G + G) % G) < c[4] &&
           (((rz - c[2]) % G + G) % G) < c[5];
}

// SEG: a batched pass over subvolumes; each chunk takes its box, cell table,
// radius and density normalisation from its subvolume's descriptor.
template <typename T, int P, bool SEG>
__global__ void __launch_bounds__(kKnnThreads, 4) knn_kernel(KnnDev<T> a)
{
    using L = WarpSmem<T, P>;
    constexpr int Q = L::Q;
    constexpr int TILE = L::TILE;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int q = lane / P, p = lane % P;
    const uint32_t gmask = (P == 32) ? FULL : (((1u << P) - 1u) << (q * P));
    const uint32_t lt_mask = (1u << lane) - 1u;

    unsigned char *wbase = smem_raw + L::total(a.buf) * wib;
    Rec<T> *tile = (Rec<T> *)(wbase + L::tile());
    T *bd = (T *)(wbase + L::bd()) + (size_t)q * a.buf;
    uint32_t *bs = (uint32_t *)(wbase + L::bs(a.buf)) + (size_t)q * a.buf;
    int *hist = (int *)(wbase + L::hist(a.buf)) + q * kHistBins;
    uint32_t *rs = (uint32_t *)(wbase + L::rs(a.buf));
    uint32_t *ro = rs + 32;     // 33 entries
    T *kthv = (T *)(wbase + L::kth(a.buf));
    T *qpos = (T *)(wbase + L::qpos(a.buf));      // Q x 3, real coordinates
    int *cube = (int *)(wbase + L::cube(a.buf));  // Q x 6: lo x3, n x3
    int *hrows = (int *)(wbase + L::hrow(a.buf));             // one padded histogram row per lane
    int *hr = hrows + lane * (kHistBins + 1);                   // this lane's row
    int *grows = hrows + q * P * (kHistBins + 1);               // the group's rows
    T *kd = (T *)(wbase + L::kd(a.buf)) + q * KCAP;
    T *od = (T *)(wbase + L::od(a.buf)) + q * OCAP;
    uint32_t *os = (uint32_t *)(wbase + L::os(a.buf)) + q * OCAP;

    const int k = a.k;
    unsigned long long cand_acc = 0, search_acc = 0, retry_acc = 0, warp_acc = 0;

    for (;;) {
        unsigned long long ch = 0;
        if (lane == 0) ch = atomicAdd(a.chunk_counter, 1ull);
        ch = __shfl_sync(FULL, ch, 0);
        if ((int64_t)ch >= a.n_chunks) break;
        ++warp_acc;
        int64_t s_first, n_end, seg_base;
        T box, half, inv_box, norm;
        const uint32_t *cellT;
        int level_dense;
        float plain_r;
        if constexpr (SEG) {
            const SegDesc &sd = a.seg[seg_of_chunk(a.seg, a.B, (int64_t)ch)];
            seg_base = sd.base;
            n_end = sd.base + sd.n;
            s_first = sd.base + ((int64_t)ch - sd.chunk0) * Q;
            box = (T)sd.box;
            half = (T)(0.5 * sd.box);
            inv_box = (T)(1.0 / sd.box);
            norm = (T)sd.norm;
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
        const typename V4<T>::type qv = a.spos[sq];
        const T rqx = qv.x, rqy = qv.y, rqz = qv.z;
        if (p == 0) {
            qpos[3 * q] = rqx;
            qpos[3 * q + 1] = rqy;
            qpos[3 * q + 2] = rqz;
        }
        __syncwarp();

        T R = a.chunk_r ? (T)a.chunk_r[ch] : (T)plain_r;
        if (!(R > T(0))) R = box * T(1e-6);
        T tau = R * R;
        int cnt = 0;
        int tbw = 0;
        bool certified = false;
        int tries = 0;

        while (!certified) {
            ++search_acc;
            // ---------------- search region for this radius: the cells of
            // the chosen level within R of some query of the chunk
            const bool full = T(2) * R >= half;
            const bool wx = __any_sync(FULL, rqx - R < T(0) || rqx + R >= box);
            const bool wy = __any_sync(FULL, rqy - R < T(0) || rqy + R >= box);
            const bool wz = __any_sync(FULL, rqz - R < T(0) || rqz + R >= box);
            // the warp's frame (x >= L/2 -> x - L on axes where some query's
            // region crosses a face) keeps every in-range difference exact
            // unless another query's region crosses L/2 on such an axis; then
            // (and for whole-box scans) each pair takes its own minimum image
            const bool mixed =
                (wx && __any_sync(FULL, rqx - R < half && half <= rqx + R)) ||
                (wy && __any_sync(FULL, rqy - R < half && half <= rqy + R)) ||
                (wz && __any_sync(FULL, rqz - R < half && half <= rqz + R));
            const bool pairwrap = full || mixed;
            const T qx = (!pairwrap && wx && rqx >= half) ? rqx - box : rqx;
            const T qy = (!pairwrap && wy && rqy >= half) ? rqy - box : rqy;
            const T qz = (!pairwrap && wz && rqz >= half) ? rqz - box : rqz;

            tau = full ? T(INFINITY) : R * R;
            cnt = 0;
            tbw = bin_base(tau);              // histogram window of this lane's row
#pragma unroll
            for (int b = 0; b < kHistBins; ++b) hr[b] = 0;
            // candidates farther than R from every query are farther than
            // R + (half-diagonal of the queries' box) from the box centre:
            // staging drops them with one distance test
            T fcx, fcy, fcz, rc2;
            {
                T lx = qx, ly = qy, lz = qz, hx = qx, hy = qy, hz = qz;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    lx = min(lx, __shfl_xor_sync(FULL, lx, o));
                    ly = min(ly, __shfl_xor_sync(FULL, ly, o));
                    lz = min(lz, __shfl_xor_sync(FULL, lz, o));
                    hx = max(hx, __shfl_xor_sync(FULL, hx, o));
                    hy = max(hy, __shfl_xor_sync(FULL, hy, o));
                    hz = max(hz, __shfl_xor_sync(FULL, hz, o));
                }
                fcx = T(0.5) * (lx + hx); fcy = T(0.5) * (ly + hy); fcz = T(0.5) * (lz + hz);
                const T ex = T(0.5) * (hx - lx), ey = T(0.5) * (hy - ly), ez = T(0.5) * (hz - lz);
                const T rc = R + sqrt(ex * ex + ey * ey + ez * ez);
                rc2 = (full || pairwrap) ? T(INFINITY) : rc * rc * T(1.0001) + box * box * T(1e-12);
            }

            int l = 1, G = 2;
            if (!full) {
                const T cells = box * (T)a.cpr / R;   // 2^l <= cells: side >= R / cpr
                while (l < kMaxLevel && (T)(1 << (l + 1)) <= cells) ++l;
                G = 1 << l;
            }
            const T sc = inv_box * (T)G;
            const T csz = box / (T)G;
            const T hcs = T(0.5) * csz;
            const T R2c = R * R * T(1.00001) + box * box * T(1e-12);
            // this query's cube of cells (unwrapped indices) and the warp's bounding cube
            const int qlx = (int)floor((rqx - R) * sc), qhx = (int)floor((rqx + R) * sc);
            const int qly = (int)floor((rqy - R) * sc), qhy = (int)floor((rqy + R) * sc);
            const int qlz = (int)floor((rqz - R) * sc), qhz = (int)floor((rqz + R) * sc);
            int blx = qlx, bly = qly, blz = qlz, bhx = qhx, bhy = qhy, bhz = qhz;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                blx = min(blx, __shfl_xor_sync(FULL, blx, o));
                bly = min(bly, __shfl_xor_sync(FULL, bly, o));
                blz = min(blz, __shfl_xor_sync(FULL, blz, o));
                bhx = max(bhx, __shfl_xor_sync(FULL, bhx, o));
                bhy = max(bhy, __shfl_xor_sync(FULL, bhy, o));
                bhz = max(bhz, __shfl_xor_sync(FULL, bhz, o));
            }
            const int64_t nbx = bhx - blx + 1, nby = bhy - bly + 1, nbz = bhz - blz + 1;
            const bool one = nbx <= G && nby <= G && nbz <= G && nbx * nby * nbz <= 1024;
            __syncwarp();
            if (p == 0) {
                int *cq = cube + 6 * q;
                cq[0] = qlx; cq[1] = qly; cq[2] = qlz;
                cq[3] = min(qhx - qlx + 1, G); cq[4] = min(qhy - qly + 1, G); cq[5] = min(qhz - qlz + 1, G);
            }
            __syncwarp();
            const int ncubes = (full || one) ? 1 : nq;

            for (int cc = 0; cc < ncubes; ++cc) {
                int c0x = 0, c0y = 0, c0z = 0, nx = 1, ny = 1, nz = 1;
                if (!full) {
                    if (one) {
                        c0x = blx; c0y = bly; c0z = blz;
                        nx = (int)nbx; ny = (int)nby; nz = (int)nbz;
                    } else {
                        const int *cq = cube + 6 * cc;
                        c0x = cq[0]; c0y = cq[1]; c0z = cq[2];
                        nx = cq[3]; ny = cq[4]; nz = cq[5];
                    }
                }
                const int ncells = full ? 1 : nx * ny * nz;
                for (int cb = 0; cb < ncells; cb += 32) {
                    // --------- one batch of up to 32 cells: ranges and prefix
                    uint32_t ra = 0, rb = 0;
                    const int ci = cb + lane;
                    if (full) {
                        if (lane == 0) { ra = (uint32_t)seg_base; rb = (uint32_t)n_end; }
                    } else if (ci < ncells) {
                        const int ix = c0x + ci % nx, iy = c0y + (ci / nx) % ny, iz = c0z + ci / (nx * ny);
                        const int rx = ((ix % G) + G) % G, ry = ((iy % G) + G) % G, rz = ((iz % G) + G) % G;
                        bool keep = true;
                        for (int c2 = 0; c2 < cc; ++c2)
                            if (in_cube(cube + 6 * c2, rx, ry, rz, G)) { keep = false; break; }
                        if (keep) {
                            // periodic distance from each query to the cell box
                            keep = false;
                            const T cx = ((T)rx + T(0.5)) * csz, cy = ((T)ry + T(0.5)) * csz,
                                    cz = ((T)rz + T(0.5)) * csz;
                            for (int j = 0; j < nq; ++j) {
                                T dx = fabs(cx - qpos[3 * j]), dy = fabs(cy - qpos[3 * j + 1]),
                                  dz = fabs(cz - qpos[3 * j + 2]);
                                dx = max(T(0), min(dx, box - dx) - hcs);
                                dy = max(T(0), min(dy, box - dy) - hcs);
                                dz = max(T(0), min(dz, box - dz) - hcs);
                                if (dx * dx + dy * dy + dz * dz <= R2c) { keep = true; break; }
                            }
                        }
                        if (keep) {
                            const uint64_t code = morton3((uint32_t)rx, (uint32_t)ry, (uint32_t)rz);
                            cell_range(cellT, a.keys, level_dense, l, code, ra, rb);
                        }
                    }
                    uint32_t len = rb - ra, inc = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        uint32_t y = __shfl_up_sync(FULL, inc, o);
                        if (lane >= o) inc += y;
                    }
                    const uint32_t total = __shfl_sync(FULL, inc, 31);
                    __syncwarp();
                    rs[lane] = ra;
                    ro[lane] = inc - len;
                    if (lane == 31) ro[32] = inc;
                    __syncwarp();

                    // --------- stream the batch's candidates through the tile.  The
                    // next tile's global loads are issued before the current tile
                    // is tested, so their latency overlaps the tests.
                    constexpr int PER_LANE = TILE / 32;
                    typename V4<T>::type pv[PER_LANE];
                    uint32_t pidx[PER_LANE];
                    int cur = 0;   // range of this lane's next element (moves forward only)
                    auto fetch = [&](uint32_t t0) {
#pragma unroll
                        for (int jj = 0; jj < PER_LANE; ++jj) {
                            const uint32_t g = t0 + (uint32_t)(lane + 32 * jj);
                            pidx[jj] = 0xffffffffu;
                            if (g < total) {
                                while (ro[cur + 1] <= g) ++cur;
                                pidx[jj] = rs[cur] + (g - ro[cur]);
                            }
                        }
#pragma unroll
                        for (int jj = 0; jj < PER_LANE; ++jj)
                            if (pidx[jj] != 0xffffffffu) pv[jj] = a.spos[pidx[jj]];
                    };
                    if (total > 0) fetch(0);
                    for (uint32_t t0 = 0; t0 < total; t0 += TILE) {
                        int m = 0;   // staged candidates that pass the chunk-sphere test
#pragma unroll
                        for (int jj = 0; jj < PER_LANE; ++jj) {
                            Rec<T> rec;
                            bool keep = false;
                            if (pidx[jj] != 0xffffffffu) {
                                const typename V4<T>::type v = pv[jj];
                                if (pairwrap) {
                                    rec.x = v.x; rec.y = v.y; rec.z = v.z;
                                } else {
                                    rec.x = (wx && v.x >= half) ? v.x - box : v.x;
                                    rec.y = (wy && v.y >= half) ? v.y - box : v.y;
                                    rec.z = (wz && v.z >= half) ? v.z - box : v.z;
                                }
                                rec.s = pidx[jj];
                                const T dx = rec.x - fcx, dy = rec.y - fcy, dz = rec.z - fcz;
                                keep = dx * dx + dy * dy + dz * dz <= rc2;
                            }
                            const uint32_t kb = __ballot_sync(FULL, keep);
                            if (keep) tile[m + __popc(kb & lt_mask)] = rec;
                            m += __popc(kb);
                        }
                        __syncwarp();
                        if (t0 + TILE < total) fetch(t0 + TILE);
                        cand_acc += (unsigned long long)m * (unsigned long long)nq;
                        // --------- test staged candidates, 4 per lane per step
                        constexpr int STEP = 4 * P;
                        const int steps = (m + STEP - 1) / STEP;
                        for (int st = 0; st < steps; ++st) {
                            T d2[4];
                            uint32_t sj[4];
                            bool ps[4];
                            int c = 0;
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int j = st * STEP + u * P + p;
                                ps[u] = false;
                                d2[u] = T(0);
                                sj[u] = 0;
                                if (j < m && active) {
                                    const Rec<T> cd = tile[j];
                                    T dx, dy, dz;
                                    if (pairwrap) {
                                        dx = wrapdiff(cd.x, rqx, box, half);
                                        dy = wrapdiff(cd.y, rqy, box, half);
                                        dz = wrapdiff(cd.z, rqz, box, half);
                                    } else {
                                        dx = cd.x - qx; dy = cd.y - qy; dz = cd.z - qz;
                                    }
                                    d2[u] = fma(dx, dx, fma(dy, dy, dz * dz));
                                    sj[u] = cd.s;
                                    ps[u] = d2[u] <= tau;
                                }
                                c += ps[u] ? 1 : 0;
                            }
                            // positions: exclusive prefix of the pass counts in the group
                            int incl = c;
#pragma unroll
                            for (int o = 1; o < P; o <<= 1) {
                                const int y = __shfl_up_sync(FULL, incl, o, P);
                                if (p >= o) incl += y;
                            }
                            const int gtot = __shfl_sync(FULL, incl, P - 1, P);
                            int pos = cnt + incl - c;
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                if (ps[u]) {
                                    bd[pos] = d2[u];
                                    bs[pos] = sj[u];
                                    ++pos;
                                    ++hr[bin_of(d2[u], tbw)];
                                }
                            }
                            cnt += gtot;
                            // --------- compaction when a buffer fills up
                            if (__any_sync(FULL, cnt > a.cap)) {
                                const bool need = cnt > a.cap;
                                const int cmax = warp_max_i(cnt);
                                int tb = tbw, bk, bo, below_k, upto_k;
                                bool rows_ok;
                                __syncwarp();
                                rows_scan<P>(need, grows, cnt, k, 0, p, gmask, bk, bo, below_k, upto_k, rows_ok);
                                if (!__all_sync(FULL, rows_ok))
                                    warp_hist<T, P>(need, bd, cnt, cmax, hist, k, 0, p, gmask, tb, bk, bo, below_k,
                                                    upto_k);
                                // the bin edge shrinks the buffer only if the k-th entry's bin
                                // is not crowded (candidates in a distant dense clump can share
                                // one bin); otherwise cut at the exact k-th value
                                T ntau = (need && bk < kHistBins - 1 && upto_k <= a.cap - 4 * P)
                                             ? bin_upper(tau, tb, bk) : T(-1);
                                const bool exact = need && !(ntau >= T(0));
                                if (__any_sync(FULL, exact)) {
                                    warp_kth<T, P>(exact, bd, cnt, cmax, hist, tb, bk, below_k, upto_k, k, p,
                                                   gmask, lt_mask, kd, &kthv[q]);
                                    if (exact) ntau = kthv[q];
                                    __syncwarp();
                                }
                                warp_compact<T, P>(need, bd, bs, cnt, cmax, ntau, p, gmask, lt_mask);
                                if (need) {
                                    tau = ntau;
                                    if (cnt > a.cap) {
                                        if (p == 0) atomicOr(a.err, kErrDegenerate);
                                        cnt = a.cap;
                                    }
                                    // rebuild this group's rows for the new window
                                    tbw = bin_base(tau);
#pragma unroll
                                    for (int b = 0; b < kHistBins; ++b) hr[b] = 0;
                                }
                                __syncwarp();
                                const int cmax2 = warp_max_i(need ? cnt : 0);
                                for (int e0 = 0; e0 < cmax2; e0 += P) {
                                    const int e = e0 + p;
                                    if (need && e < cnt) ++hr[bin_of(bd[e], tbw)];
                                }
                            }
                        }
                        __syncwarp();
                    }
                }
            }
            // ---------------- certification
            const bool ok = !active || cnt >= k;
            if (__all_sync(FULL, ok)) {
                certified = true;
            } else {
                ++retry_acc;
                if (++tries >= kMaxTries || full) {
                    if (lane == 0) atomicOr(a.err, kErrKnnRetry);
                    break;
                }
                T f = T(1.25);
                if (!ok) {
                    T need = T(1.1) * cbrt((T)k / (T)max(cnt, 1));
                    f = max(f, need);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) f = max(f, __shfl_xor_sync(FULL, f, o));
                R *= min(f, T(8));
            }
        }
        if (!certified) continue;

        // -------------------- selection (all lanes, per query group)
        {
            const bool need = active;
            const int n_out = (a.nbr_s != nullptr) ? a.n_out : 0;
            const int cmax = warp_max_i(cnt);
            int tb = tbw, bk, bo, below_k, upto_k;
            bool rows_ok;
            __syncwarp();
            rows_scan<P>(need, grows, cnt, k, n_out, p, gmask, bk, bo, below_k, upto_k, rows_ok);
            if (!__all_sync(FULL, rows_ok))
                warp_hist<T, P>(need, bd, cnt, cmax, hist, k, n_out, p, gmask, tb, bk, bo, below_k, upto_k);
            // one pass gathers the k-th entry's bin (for the exact r_k) and
            // the entries up to the n_out-th entry's bin (for the list)
            int nk = 0, no = 0;
            for (int e0 = 0; e0 < cmax; e0 += P) {
                const int e = e0 + p;
                T v = T(0);
                bool ink = false, ino = false;
                if (need && e < cnt) {
                    v = bd[e];
                    const int b = bin_of(v, tb);
                    ink = b == bk;
                    ino = n_out > 0 && b <= bo;
                }
                const uint32_t mk = __ballot_sync(FULL, ink) & gmask;
                const uint32_t mo = __ballot_sync(FULL, ino) & gmask;
                if (ink) {
                    const int pos = nk + __popc(mk & lt_mask);
                    if (pos < KCAP) kd[pos] = v;
                }
                if (ino) {
                    const int pos = no + __popc(mo & lt_mask);
                    if (pos < OCAP) { od[pos] = v; os[pos] = bs[e]; }
                }
                nk += __popc(mk);
                no += __popc(mo);
            }
            __syncwarp();
            {
                const bool small = nk <= KCAP;
                const int nkmax = warp_max_i((need && small) ? nk : 0);
                for (int e0 = 0; e0 < nkmax; e0 += P) {
                    const int e = e0 + p;
                    const bool mine = need && small && e < nk;
                    const T v = mine ? kd[e] : T(0);
                    int lt = below_k, le = below_k;
                    for (int f = 0; f < nkmax; ++f) {
                        if (f < nk) {
                            const T u = kd[f];
                            lt += u < v;
                            le += u <= v;
                        }
                    }
                    if (mine && lt < k && k <= le) kthv[q] = v;
                }
                __syncwarp();
                if (__any_sync(FULL, need && !small && bk > 0))
                    warp_kth_deep<T, P>(need && !small && bk > 0, bd, cnt, cmax, hist, tb, bk, below_k, upto_k, k,
                                        p, gmask, lt_mask, kd, &kthv[q]);
                if (__any_sync(FULL, need && !small && bk == 0)) {
                    for (int e0 = 0; e0 < cmax; e0 += P) {
                        const int e = e0 + p;
                        if (!(need && !small && bk == 0 && e < cnt)) continue;
                        const T v = bd[e];
                        if (bin_of(v, tb) != bk) continue;
                        int lt = below_k, le = below_k;
                        for (int f = 0; f < cnt; ++f) {
                            const T u = bd[f];
                            if (bin_of(u, tb) != bk) continue;
                            lt += u < v;
                            le += u <= v;
                        }
                        if (lt < k && k <= le) kthv[q] = v;
                    }
                }
                __syncwarp();
            }
            const T vk = kthv[q];
            // density: fixed-point sum of w(2 r / r_k) over entries with d^2 < r_k^2
            unsigned long long wsum = 0;
            const T rk = sqrt(vk);
            const T inv_h = vk > T(0) ? T(2) / rk : T(0);
            for (int e0 = 0; e0 < cmax; e0 += P) {
                const int e = e0 + p;
                if (need && e < cnt) {
                    const T v = bd[e];
                    if (v < vk) {
                        const T w = m4<T>(sqrt(v) * inv_h);
                        wsum += (unsigned long long)(w * T(4294967296.0) + T(0.5));
                    }
                }
            }
#pragma unroll
            for (int o = 1; o < P; o <<= 1) wsum += __shfl_xor_sync(FULL, wsum, o);
            // the n_out nearest in (d^2, original index) order, ranked in the
            // small list (the whole buffer only when that list overflowed)
            if (n_out > 0) {
                const bool small = no <= OCAP;
                const int nomax = warp_max_i((need && small) ? no : 0);
                for (int e0 = 0; e0 < nomax; e0 += P) {
                    const int e = e0 + p;
                    const bool mine = need && small && e < no;
                    const T v = mine ? od[e] : T(0);
                    const uint32_t se = mine ? os[e] : 0u;
                    uint32_t oe = 0xffffffffu;
                    int rank = 0;
                    for (int f = 0; f < nomax; ++f) {
                        if (f < no) {
                            const T u = od[f];
                            rank += u < v;
                            if (mine && u == v && f != e) {
                                if (oe == 0xffffffffu) oe = orig_of<T>(a.spos[se]);
                                rank += orig_of<T>(a.spos[os[f]]) < oe;
                            }
                        }
                    }
                    if (mine && rank < n_out) a.nbr_s[(size_t)sq * a.ld_out + rank] = se;
                }
                if (__any_sync(FULL, need && !small)) {
                    for (int e0 = 0; e0 < cmax; e0 += P) {
                        const int e = e0 + p;
                        if (!(need && !small && e < cnt)) continue;
                        const T v = bd[e];
                        if (bin_of(v, tb) > bo) continue;
                        const uint32_t se = bs[e];
                        uint32_t oe = 0xffffffffu;
                        int rank = 0;
                        for (int f = 0; f < cnt; ++f) {
                            const T u = bd[f];
                            if (u < v) { ++rank; continue; }
                            if (u == v && f != e) {
                                if (oe == 0xffffffffu) oe = orig_of<T>(a.spos[se]);
                                rank += orig_of<T>(a.spos[bs[f]]) < oe;
                            }
                        }
                        if (rank < n_out) a.nbr_s[(size_t)sq * a.ld_out + rank] = se;
                    }
                }
            }
            if (need && p == 0) {
                float dens;
                if (vk > T(0)) {
                    const T h = rk * T(0.5);
                    dens = (float)(norm * ((T)wsum * T(2.3283064365386963e-10)) / (h * h * h));
                } else {
                    dens = INFINITY;
                }
                a.dens_s[sq] = dens;
                if (a.rk_s) a.rk_s[sq] = (float)rk;
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

template <typename T, int P> size_t knn_smem_per_warp(int buf) { return WarpSmem<T, P>::total(buf); }

template <typename T, int P, bool SEG> int knn_run(hop_ctx *c, const KnnArgs &a, int cpr)
{
    constexpr int Q = 32 / P;
    KnnDev<T> d;
    d.spos = (const typename V4<T>::type *)a.spos;
    d.keys = a.keys;
    d.cellT = a.cellT;
    d.level_dense = a.level_dense;
    d.n = a.n;
    d.n_chunks = SEG ? a.n_chunks : (a.n + Q - 1) / Q;
    d.seg = a.seg;
    d.B = a.B;
    d.box = (T)a.box;
    d.inv_box = (T)(1.0 / a.box);
    d.half_box = (T)(0.5 * a.box);
    d.k = a.k;
    d.n_out = a.n_out;
    d.ld_out = a.ld_out;
    // room for 4 Ndens entries per query (3 with 8 or more queries per warp,
    // where the larger buffer would cost a resident block): compactions are
    // rare.  A tuned context may set 2, 3 or 4.
    d.cap = (c->capf ? c->capf : (Q <= 4 ? 4 : 3)) * a.k;
    d.buf = d.cap + 4 * P + 4;
    d.chunk_r = a.chunk_r;
    d.plain_r = a.plain_r;
    d.cpr = cpr;
    d.norm = (T)(a.box * a.box * a.box / ((double)(a.n_norm > 0 ? a.n_norm : a.n) * 3.14159265358979323846));
    d.nbr_s = a.nbr_s;
    d.dens_s = a.dens_s;
    d.rk_s = a.rk_s;
    d.counters = c->d_counters;
    d.chunk_counter = c->d_counters + kCntNum;
    d.err = c->d_err;
    HOP_CUDA(c, cudaMemsetAsync(d.chunk_counter, 0, sizeof(unsigned long long), c->stream));
    // as many warps per block (4, 2 or 1) as fit in the opt-in shared memory
    int max_smem = 0;
    HOP_CUDA(c, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    const size_t per_warp = knn_smem_per_warp<T, P>(d.buf);
    int warps = kKnnWarps;
    while (warps > 1 && per_warp * warps > (size_t)max_smem) warps >>= 1;
    if (per_warp * warps > (size_t)max_smem)
        return ctx_fail(c, HOP_EINVAL, "kNN search buffer does not fit in shared memory");
    const size_t smem = per_warp * warps;
    auto kern = knn_kernel<T, P, SEG>;
    HOP_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    HOP_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
    if (per_sm < 1) return ctx_fail(c, HOP_EINVAL, "kNN search buffer does not fit in shared memory");
    int64_t blocks = (int64_t)per_sm * c->num_sms;
    const int64_t need = (d.n_chunks + warps - 1) / warps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, warps * 32, smem, c->stream>>>(d);
    HOP_LAUNCH(c);
    return HOP_OK;
}

}  // namespace

int knn_launch(hop_ctx *c, const KnnArgs &a, bool f64, int qpw, int cpr)
{
    if (a.k < 2 || a.k > kMaxDens) return ctx_fail(c, HOP_EINVAL, "n_dens out of range");
    if (cpr < 1 || cpr > 4) cpr = 1;
    if (qpw == 32 && !f64) return knn32_launch(c, a, cpr);   // one query per lane
    // float32 with 4, 8 or 16 queries per warp: the count-then-gather kernel,
    // unless a candidate-buffer factor was set (the single-scan kernel below)
    if (!f64 && c->capf == 0 && (qpw == 4 || qpw == 8 || qpw == 16)) return knn_cg_launch(c, a, qpw, cpr);
    if (a.seg) {
        // batched passes: float32 positions, 4, 8, 16 or 32 queries per warp
        if (f64) return ctx_fail(c, HOP_EINVAL, "batched passes take float32 positions");
        switch (qpw) {
        case 16: return knn_run<float, 2, true>(c, a, cpr);
        case 8: return knn_run<float, 4, true>(c, a, cpr);
        case 4: return knn_run<float, 8, true>(c, a, cpr);
        default: return ctx_fail(c, HOP_EINVAL, "batched passes take 4, 8, 16 or 32 queries per warp");
        }
    }
    switch (qpw) {
    case 32: return f64 ? knn_run<double, 1, false>(c, a, cpr) : knn_run<float, 1, false>(c, a, cpr);
    case 16: return f64 ? knn_run<double, 2, false>(c, a, cpr) : knn_run<float, 2, false>(c, a, cpr);
    case 8: return f64 ? knn_run<double, 4, false>(c, a, cpr) : knn_run<float, 4, false>(c, a, cpr);
    case 4: return f64 ? knn_run<double, 8, false>(c, a, cpr) : knn_run<float, 8, false>(c, a, cpr);
    case 2: return f64 ? knn_run<double, 16, false>(c, a, cpr) : knn_run<float, 16, false>(c, a, cpr);
    case 1: return f64 ? knn_run<double, 32, false>(c, a, cpr) : knn_run<float, 32, false>(c, a, cpr);
    default: return ctx_fail(c, HOP_EINVAL, "queries per warp must be 1, 2, 4, 8, 16 or 32");
    }
}
