// Internal declarations of libhop: context, scratch arena, device helpers and
// the launch functions each translation unit provides.  Nothing here is part
// of the C ABI (include/hop.h is).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hop.h"

// ---------------------------------------------------------------- limits --
// Morton keys hold 16 bits per axis (48-bit keys): levels 0..16 of the
// octree over the box; level l has 2^l cells per axis.
constexpr int kMaxLevel = 16;
constexpr int kMaxDens = 128;    // Ndens limit (search buffer is 4 * Ndens + slack)
constexpr int kHistBins = 32;    // 1/8-octave bins of d^2 used for selection

// Device error word bits (atomicOr'ed by kernels, read by the host).
enum : uint32_t {
    kErrBadPos = 1u << 0,       // a coordinate outside [0, box) or NaN
    kErrKnnRetry = 1u << 1,     // kNN search ran out of retries
    kErrDegenerate = 1u << 2,   // more equidistant neighbours than the buffer holds
    kErrChainLoop = 1u << 3,    // chain following hit its iteration limit
    kErrTableFull = 1u << 4,    // boundary hash table overflow
    kErrMergeLoop = 1u << 5,    // merge rounds hit their limit
    kErrBadIndex = 1u << 6,     // an index array holds a value >= n
    kErrChainCap = 1u << 7,     // more chains above delta_outer than a batched pass's merge arrays hold
    kErrSortWait = 1u << 8,     // a radix pass's look-back wait hit its limit
};

// Scratch slots owned by a context.  Each slot grows on demand.
enum Slot {
    S_POS_IN,      // device copy of host positions
    S_KEY0, S_KEY1, S_VAL0, S_VAL1,   // radix sort ping-pong
    S_SORT_TMP,    // per-block digit counts of the radix sort
    S_SCAN,        // partial sums of the device-wide scan
    S_SPOS,        // sorted positions (float4 / double4): x, y, z, original index
    S_CELLT,       // cell start table at the dense level
    S_CHUNK_R,     // per-chunk first search radius
    S_CHUNK_LVL,   // per-chunk feature level (u8) / scratch
    S_NBR_S,       // neighbour lists in sorted order (sorted indices)
    S_DENS_S,      // densities in sorted order
    S_RK_S,        // r_k in sorted order
    S_DKEY,        // (density bits << 32) | ~original index
    S_HOP, S_CHAIN,
    S_HKEY, S_HVAL, // boundary hash table
    S_EDGE_KEY, S_EDGE_SUM, S_EDGE_TMP,
    S_MERGE,       // merge arrays (chains, components, ranks ...)
    S_GROUP_S,
    S_MISC,
    S_MLP_TMP,
    S_OUT_DENS, S_OUT_GROUP,            // device staging of host outputs
    S_GROUP_OUT,                        // group ids in sorted order
    S_ESORT_K0, S_ESORT_K1, S_ESORT_V0, S_ESORT_V1, S_ESORT_TMP,   // edge-list sort
    S_SEG,                              // subvolume descriptors of a batched pass
    S_BATCH,                            // per-pass arrays of a batched pass
    S_HALO,                             // halo statistics scratch
    S_SUB,                              // subhalos: dense chain ids, per-particle chain ids
    S_SUB_C,                            // subhalos: arrays over chains and boundaries
    S_COUNT
};

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct MlpState {
    bool loaded = false;
    float *w32 = nullptr;      // fp32 master parameters (device)
    uint16_t *w16 = nullptr;   // bf16 copy used by every forward pass (device)
    float *m = nullptr, *v = nullptr, *g = nullptr;   // Adam moments, gradient
    float log_margin = 0.f;
    int64_t step = 0;
};

struct hop_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::string err;
    DevBuf buf[S_COUNT];
    uint32_t *d_err = nullptr;          // device error word
    unsigned long long *d_counters = nullptr;   // kNN counters (see kCnt*)
    void *h_pinned = nullptr;           // small pinned host staging area
    hop_stats stats{};
    int64_t launches = 0;               // kernels launched (all calls)
    MlpState mlp_bank[6];               // one network per queries-per-warp setting
    MlpState *mlp = mlp_bank + 3;       // the network of the current setting
    int qpw = 8;                        // kNN queries per warp
    int cpr = 1;                        // search cells per radius
    int capf = 0;                       // kNN kernel choice: 0 count-then-gather, 2-6 single-scan buffer in Ndens
    int64_t norm_n = 0;                 // hop_set_norm_count: density normalisation count (0: n of the call)
    // graph capture of the batched pass
    bool capturing = false;             // a capture is open on `stream`
    std::vector<void *> graveyard;      // buffers replaced while capturing, freed with the graph
    uint64_t buf_epoch = 0;             // bumped whenever a slot's buffer moves
    struct BatchGraph *batch = nullptr; // cached graph of the last batched pass
    cudaStream_t side = nullptr;        // capture stream of loop bodies
    cudaStream_t cap = nullptr;         // capture stream of a pass (the caller's may be the legacy stream)
    // sorted state of the last density pass (for hop_mlp_samples)
    int64_t last_n = 0;
    int last_level_dense = 0;
    int last_qpw = 8;
    double last_box = 1.0;
    bool last_f64 = false;
    int last_ndens = 0;
    const void *last_spos = nullptr;
    const uint64_t *last_keys = nullptr;
    const uint32_t *last_cellT = nullptr;
    const float *last_rk = nullptr;
    cudaEvent_t ev[12] = {};
};

inline int qpw_index(int qpw)
{
    int i = 0;
    while (i < 5 && (1 << i) < qpw) ++i;
    return i;
}

// Counters slot indices in d_counters.
enum { kCntCand = 0, kCntSearch, kCntRetry, kCntWarps, kCntQual, kCntEdges, kCntNum };

// ------------------------------------------------------ host-side helpers --
int ctx_fail(hop_ctx *c, int code, const std::string &msg);
int ctx_cuda(hop_ctx *c, cudaError_t e, const char *what);
void *ctx_buf(hop_ctx *c, Slot s, size_t bytes);   // nullptr on failure (err set)
int ctx_check_device_error(hop_ctx *c);            // syncs; maps the error word

#define HOP_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ctx_cuda((ctx), e_, #call); \
    } while (0)

#define HOP_LAUNCH(ctx)                                           \
    do {                                                          \
        ++(ctx)->launches;                                        \
        cudaError_t e_ = cudaGetLastError();                      \
        if (e_ != cudaSuccess) return ctx_cuda((ctx), e_, "kernel launch"); \
    } while (0)

// ------------------------------------------------------ device helpers ---

// Morton code of cell (x, y, z), coordinates below 2^16: bit i of x, y and
// z goes to bit 3i, 3i + 1 and 3i + 2.  The bits are spread on 8-bit halves
// in 32-bit arithmetic: bits 0-7 of the coordinates fill bits 0-23 of the
// code, bits 8-15 fill bits 24-47.
__host__ __device__ inline uint32_t spread3_8(uint32_t v)
{
    v &= 0xFFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__host__ __device__ inline uint64_t morton3(uint32_t x, uint32_t y, uint32_t z)
{
    const uint32_t lo = spread3_8(x) | (spread3_8(y) << 1) | (spread3_8(z) << 2);
    const uint32_t hi = spread3_8(x >> 8) | (spread3_8(y >> 8) << 1) | (spread3_8(z >> 8) << 2);
    return ((uint64_t)hi << 24) | lo;
}

// Level of the dense cell table for n particles: the first level with at
// least n cells, plus one (so deeper cells, found by binary search, hold few
// particles), at most level 10 (2^30 cells, a 4 GB table).
inline int dense_level_for(int64_t n)
{
    int l = 1;
    while (l < 10 && (int64_t(1) << (3 * l)) < n) ++l;
    return l < 10 ? l + 1 : 10;
}

// First search radius of the plain path: the distance of the k-th nearest
// neighbour at the box's mean density, the radius of a ball that holds k of
// the n particles on average: (3 k L^3 / (4 pi n))^(1/3).  The certified
// search expands it where the ball holds fewer than k.
inline float plain_radius_for(int64_t n, double box, int k)
{
    const double r = box * cbrt(3.0 * (double)k / (4.0 * 3.14159265358979323846 * (double)n));
    return (float)r;
}

// ------------------------------------------------------------ batches ----
// One subvolume of a batched pass.  Its particles are the contiguous range
// [base, base + n) both in the caller's order and after the sort (the sort
// key leads with the subvolume number); its query chunks are
// [chunk0, chunk0 + ceil(n / Q)); its dense cell table (level level_dense,
// entries holding global sorted positions) starts at cell0.
struct SegDesc {
    int64_t base, n, chunk0, cell0;
    double box;
    double norm;          // box^3 / (n pi): density normalisation
    float plain_r;
    int level_dense;
};

// The subvolume holding chunk `ch`: the last b with seg[b].chunk0 <= ch.
__device__ __forceinline__ int seg_of_chunk(const SegDesc *__restrict__ seg, int B, int64_t ch)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (seg[m].chunk0 <= ch) lo = m; else hi = m - 1;
    }
    return lo;
}

// The subvolume holding particle `i` (caller's or sorted order).
__device__ __forceinline__ int seg_of_index(const SegDesc *__restrict__ seg, int B, int64_t i)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (seg[m].base <= i) lo = m; else hi = m - 1;
    }
    return lo;
}

// Grid for a grid-stride loop over n items: 256-thread blocks, at most 32
// blocks per SM, at least one block.
inline int grid_for(hop_ctx *c, int64_t n)
{
    int64_t b = (n + 255) / 256;
    b = b < (int64_t)c->num_sms * 32 ? b : (int64_t)c->num_sms * 32;
    return (int)(b > 1 ? b : 1);
}

// Offsets of arrays packed into one scratch buffer start on 256 bytes.
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Density keys: (density bits << 32) | (0xFFFFFFFF - original index).
__device__ __forceinline__ float key_dens(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ uint32_t key_orig(uint64_t k) { return 0xFFFFFFFFu - (uint32_t)k; }

// Root of x in a union-find forest whose parents only point to smaller
// labels (so every walk ends); the walk is bounded all the same.
__device__ __forceinline__ uint32_t find_root(const uint32_t *parent, uint32_t x)
{
    for (int g = 0; g < (1 << 24); ++g) {
        const uint32_t p = parent[x];
        if (p == x) return x;
        x = p;
    }
    return x;
}

// Warp aggregation for per-group atomics: `peers` is the set of lanes that
// hold the same group (__match_any_sync); every lane of the set gets the
// sum or maximum of the set's values, combined in ascending lane order.
__device__ __forceinline__ long long peer_sum_ll(uint32_t peers, long long v)
{
    long long s = 0;
    for (uint32_t m = peers; m; m &= m - 1) s += __shfl_sync(peers, v, __ffs(m) - 1);
    return s;
}
__device__ __forceinline__ double peer_sum_f64(uint32_t peers, double v)
{
    double s = 0.0;
    for (uint32_t m = peers; m; m &= m - 1) s += __shfl_sync(peers, v, __ffs(m) - 1);
    return s;
}
__device__ __forceinline__ unsigned long long peer_max(uint32_t peers, unsigned long long v)
{
    unsigned long long b = 0;
    for (uint32_t m = peers; m; m &= m - 1) {
        const unsigned long long u = __shfl_sync(peers, v, __ffs(m) - 1);
        b = u > b ? u : b;
    }
    return b;
}

// Runs of consecutive lanes with the same group key g (each run reduced by
// one atomic): heads has a bit for every lane that starts a run.
__device__ __forceinline__ uint32_t run_heads(int64_t g, int lane)
{
    const int64_t prev = __shfl_up_sync(0xffffffffu, g, 1);
    return __ballot_sync(0xffffffffu, lane == 0 || prev != g);
}

// After it, the head of each run holds the sum (or maximum) of the run's
// values: a suffix scan over the run in five shuffle steps, adding lane + d
// while no run starts in (lane, lane + d].
template <typename V> __device__ __forceinline__ V run_sum(uint32_t heads, int lane, V v)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const V o = __shfl_down_sync(0xffffffffu, v, d);
        const uint32_t between = lane + d < 32 ? ((2u << (lane + d)) - (2u << lane)) : 0u;
        if (lane + d < 32 && (heads & between) == 0) v += o;
    }
    return v;
}
__device__ __forceinline__ unsigned long long run_max(uint32_t heads, int lane, unsigned long long v)
{
    if (heads == 1u) {
        // the warp is one run: two 32-bit reductions (high half, then the
        // low half among the lanes holding the highest)
        const unsigned hi = (unsigned)(v >> 32);
        const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
        const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? (unsigned)v : 0u);
        return ((unsigned long long)mh << 32) | ml;
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, v, d);
        const uint32_t between = lane + d < 32 ? ((2u << (lane + d)) - (2u << lane)) : 0u;
        if (lane + d < 32 && (heads & between) == 0 && o > v) v = o;
    }
    return v;
}
// run_sum of integers below 2^42 in magnitude; a warp that is one run sums
// the value's high part (v >> 16) and low 16 bits in two 32-bit reductions.
__device__ __forceinline__ long long run_sum_i42(uint32_t heads, int lane, long long v)
{
    if (heads == 1u)
        return ((long long)__reduce_add_sync(0xffffffffu, (int)(v >> 16)) << 16) +
               (long long)__reduce_add_sync(0xffffffffu, (unsigned)v & 0xffffu);
    return run_sum<long long>(heads, lane, v);
}
// Lanes in the run that starts at this head lane.
__device__ __forceinline__ int run_len(uint32_t heads, int lane)
{
    const uint32_t after = lane < 31 ? heads >> (lane + 1) : 0u;
    return after ? __ffs(after) : 32 - lane;
}

// A size known only on the device (an edge or chain count): kernels read
// *dev when it is set, so a captured graph needs no host round trip; `max`
// bounds it and sizes the grid.
struct DevCount {
    int64_t max;
    const uint32_t *dev;
    __device__ __forceinline__ int64_t get() const
    {
        if (!dev) return max;
        const int64_t v = (int64_t)*dev;
        return v < max ? v : max;
    }
};

// ------------------------------------------------------------ launches ---
// sort.cu
int scan_exclusive_u32(hop_ctx *c, const uint32_t *in, uint32_t *out, int64_t n,
                       uint32_t *total_dev);
int scan_exclusive_u32_dev(hop_ctx *c, const uint32_t *in, uint32_t *out, DevCount n,
                           uint32_t *total_dev);
size_t radix_sort_scratch_bytes(int64_t n);
int radix_sort_u64_dev(hop_ctx *c, uint64_t *&keys, uint64_t *&keys_alt, uint32_t *&vals,
                       uint32_t *&vals_alt, DevCount n, int begin_bit, int end_bit, void *scratch);
int radix_sort_u64(hop_ctx *c, uint64_t *&keys, uint64_t *&keys_alt, uint32_t *&vals,
                   uint32_t *&vals_alt, int64_t n, int begin_bit, int end_bit, void *scratch);
int iota_u32(hop_ctx *c, uint32_t *out, int64_t n);

// grid.cu
int grid_build(hop_ctx *c, const void *pos, int64_t n, const hop_params *p,
               void **spos_out, uint32_t **perm_out, uint64_t **keys_out, uint32_t **cellT_out,
               int *level_dense_out);
int chunk_radius(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
                 int level_dense, int64_t n, const hop_params *p, int qpw, float *chunk_r);
int chunk_features(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
                   int level_dense, int64_t n, bool f64, double box, int qpw, float *feat,
                   uint8_t *lvl, const float *rk_s, float *target);

// grid.cu, mlp.cu: batched pass (subvolume descriptors on the device)
int grid_build_seg(hop_ctx *c, const float *pos, int64_t n, const SegDesc *seg, int B,
                   int64_t n_cells, void **spos_out, uint32_t **perm_out, uint64_t **keys_out,
                   uint32_t **cellT_out);
int chunk_radius_seg(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
                     const SegDesc *seg, int B, int64_t n_chunks, int qpw, int k, float *chunk_r);
int mlp_radius_seg(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
                   const SegDesc *seg, int B, int64_t n_chunks, int qpw, int k, float *chunk_r);
// mlp.cu: the closed-form first radius of every chunk (float32 positions),
// from the same stencil counts as the learned one.
int radius_closed(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT, int Ld, int64_t n,
                  int64_t n_chunks, int qpw, double box, const SegDesc *seg, int B, int k, float log_margin,
                  float *chunk_r);

// knn.cu
struct KnnArgs {
    const void *spos;          // sorted positions (float4 / double4)
    const uint64_t *keys;      // sorted Morton keys
    const uint32_t *cellT;     // dense cell table
    int level_dense;
    int64_t n;
    double box;
    int k;                     // Ndens
    int n_out;                 // list entries written per particle
    int ld_out;                // row stride of nbr_s
    const float *chunk_r;      // per-chunk first radius, or nullptr
    float plain_r;             // first radius when chunk_r is null
    uint32_t *nbr_s;           // n x ld_out sorted indices, or nullptr
    float *dens_s;             // n
    float *rk_s;               // n or nullptr
    int64_t n_norm = 0;             // particle count of the density normalisation (0: n)
    const SegDesc *seg = nullptr;   // batched pass: subvolume descriptors (device)
    int B = 0;                      // number of subvolumes
    int64_t n_chunks = 0;           // batched pass: total query chunks
};
int knn_launch(hop_ctx *c, const KnnArgs &a, bool f64, int qpw, int cpr);
int knn32_launch(hop_ctx *c, const KnnArgs &a, int cpr);   // knn32.cu: one query per lane, float32
// knn_cg.cu: count-then-gather, float32, 4, 8 or 16 queries per warp
int knn_cg_launch(hop_ctx *c, const KnnArgs &a, int qpw, int cpr);

// link.cu
int make_dkey(hop_ctx *c, const float *dens, const uint32_t *orig, int64_t n, uint64_t *dkey);
int hop_links(hop_ctx *c, const uint64_t *dkey, const uint32_t *nbr, int ld, int64_t n, int n_hop,
              uint32_t *hop, uint32_t *chain);
// symmetric: only pairs whose chains link each other in both directions
// (ADAPTAHOP), each with the larger of the two directions' sums.
int boundaries_table(hop_ctx *c, const uint32_t *chain, const uint64_t *dkey, const uint32_t *nbr,
                     int ld, int64_t n, int n_merge, float delta_outer,
                     uint64_t **edge_key, double **edge_sum, int64_t *n_edges, bool symmetric = false);
int hop_links_async(hop_ctx *c, const uint64_t *dkey, const uint32_t *nbr, int ld, int64_t n,
                    int n_hop, uint32_t *hop, uint32_t *chain);
// The largest sum per pair of a list of (pair, sum) boundaries with
// repeated pairs (tables gathered from several subvolumes).
int edges_max_table(hop_ctx *c, const uint64_t *pair, const double *sum, int64_t m, uint64_t **edge_key,
                    double **edge_sum, int64_t *n_edges);
int boundaries_table_async(hop_ctx *c, const uint32_t *chain, const uint64_t *dkey,
                           const uint32_t *nbr, int ld, int64_t n, int n_merge, float delta_outer,
                           int64_t cap, uint32_t *m_dev, unsigned long long *nins,
                           uint64_t **edge_key, double **edge_sum);
int gather_f64(hop_ctx *c, const double *src, const uint32_t *idx, int64_t n, double *dst);
int scatter_outputs(hop_ctx *c, const uint32_t *perm, int64_t n, const float *dens_s, float *dens,
                    const int32_t *group_s, int32_t *group, const uint32_t *nbr_s, int ld_s,
                    uint32_t *nbr, int ld, int n_cols, const uint32_t *chain_s, uint32_t *chain);

// merge.cu
struct MergeGraphArgs {
    const uint32_t *chain;      // n chain labels (sorted order)
    const uint64_t *dkey;       // n density keys
    int64_t n;
    const uint64_t *edge_key;   // boundary pairs, count on the device
    const double *edge_sum;
    DevCount m;                 // edge count (max = table capacity)
    float d_o, d_s, d_p;
    const SegDesc *seg;         // subvolumes (device), B >= 1
    int B;
    int32_t *group;             // n: group rank within the subvolume, -1 = none
    uint32_t *n_groups;         // B (device): groups per subvolume
    uint32_t *counts;           // 8 device words: chains, groups, loop flag, rounds (2)
    int64_t c_cap = 0;          // chains above delta_outer the merge arrays hold (0: n); more sets kErrChainCap
};
int merge_groups_graph(hop_ctx *c, const MergeGraphArgs &a);

// batch.cu: a device-bounded loop.  Captured, it becomes a conditional
// while node whose body `body` enqueues; otherwise the host repeats it.
// The body sets *changed (a device word, zero on entry) to ask for another
// round; more than max_rounds rounds set err_bit in the error word.
void batch_free(hop_ctx *c);   // drops the cached graph and its buffers
int graph_while(hop_ctx *c, uint32_t *changed, uint32_t *round, int max_rounds, uint32_t err_bit,
                int (*body)(hop_ctx *, void *), void *arg);

int merge_groups(hop_ctx *c, const uint32_t *chain, const uint64_t *dkey, int64_t n,
                 const uint64_t *edge_key, const double *edge_sum, int64_t n_edges,
                 float delta_outer, float delta_saddle, float delta_peak,
                 int32_t *group, int64_t *n_groups);

// mlp.cu
int mlp_ensure(hop_ctx *c);
int mlp_forward_dev(hop_ctx *c, const float *feat, int64_t m, float *out);
void mlp_free(hop_ctx *c);
int mlp_radius(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
               int level_dense, int64_t n, const hop_params *p, int qpw, float *chunk_r);
