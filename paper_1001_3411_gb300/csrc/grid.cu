// Cell-grid build: Morton keys, radix sort, sorted float4 gather and the
// dense cell table (the GPU counterpart of the kD-tree build and its
// "resorted" position copy, Parallel HOP Sec. 4 "kD-tree Speedup"), plus
// per-chunk stencil counts used to pick first search radii.
#include "hop_internal.cuh"
#include "chunk_stencil.cuh"

#include <math.h>

namespace {

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4; };

__device__ __forceinline__ float4 make_rec(float x, float y, float z, uint32_t o)
{
    return make_float4(x, y, z, __uint_as_float(o));
}
__device__ __forceinline__ double4 make_rec(double x, double y, double z, uint32_t o)
{
    return make_double4(x, y, z, __longlong_as_double((long long)o));
}

template <typename T>
__global__ void keys_kernel(const T *__restrict__ pos, int64_t n, T box, T inv_box,
                            uint64_t *__restrict__ keys, uint32_t *__restrict__ idx,
                            uint32_t *__restrict__ err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        const bool ok = x >= T(0) && x < box && y >= T(0) && y < box && z >= T(0) && z < box;
        if (!ok) {
            atomicOr(err, kErrBadPos);
            x = y = z = T(0);
        }
        const uint32_t qx = min((uint32_t)(x * inv_box * T(65536)), 65535u);
        const uint32_t qy = min((uint32_t)(y * inv_box * T(65536)), 65535u);
        const uint32_t qz = min((uint32_t)(z * inv_box * T(65536)), 65535u);
        keys[i] = morton3(qx, qy, qz);
        idx[i] = (uint32_t)i;
    }
}

// Batched pass: the key leads with the subvolume number (bits 48..63), so
// one sort orders particles by subvolume, then by Morton key in its own box.
template <typename T>
__global__ void keys_seg_kernel(const T *__restrict__ pos, int64_t n, const SegDesc *__restrict__ seg,
                                int B, uint64_t *__restrict__ keys, uint32_t *__restrict__ idx,
                                uint32_t *__restrict__ err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = seg_of_index(seg, B, i);
        const double bd = seg[b].box;
        const T box = (T)bd, inv_box = (T)(1.0 / bd);
        T x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        const bool ok = x >= T(0) && x < box && y >= T(0) && y < box && z >= T(0) && z < box;
        if (!ok) {
            atomicOr(err, kErrBadPos);
            x = y = z = T(0);
        }
        const uint32_t qx = min((uint32_t)(x * inv_box * T(65536)), 65535u);
        const uint32_t qy = min((uint32_t)(y * inv_box * T(65536)), 65535u);
        const uint32_t qz = min((uint32_t)(z * inv_box * T(65536)), 65535u);
        keys[i] = ((uint64_t)b << 48) | morton3(qx, qy, qz);
        idx[i] = (uint32_t)i;
    }
}

// Sorted float4 records; with kout set, also the sorted keys without the
// subvolume field (the Morton key within the particle's own box).
template <typename T>
__global__ void gather_kernel(const T *__restrict__ pos, const uint32_t *__restrict__ perm,
                              int64_t n, typename V4<T>::type *__restrict__ spos,
                              const uint64_t *__restrict__ kin, uint64_t *__restrict__ kout)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = perm[s];
        spos[s] = make_rec(pos[3 * (int64_t)p], pos[3 * (int64_t)p + 1], pos[3 * (int64_t)p + 2], p);
        if (kout) kout[s] = kin[s] & ((uint64_t(1) << 48) - 1);
    }
}

// Every lane holds a run t[lo, hi) to fill with v (empty when !act).  Runs
// of up to 32 entries are written by their lane; longer ones (the empty
// cells of voids) by the whole warp, 32 consecutive entries per store.
__device__ __forceinline__ void fill_runs(uint32_t *t, int64_t lo, int64_t hi, uint32_t v, bool act)
{
    const unsigned lane = threadIdx.x & 31u;
    const bool big = act && hi - lo > 32;
    if (act && !big)
        for (int64_t c = lo; c < hi; ++c) t[c] = v;
    unsigned m = __ballot_sync(0xffffffffu, big);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        uint32_t *tt = (uint32_t *)__shfl_sync(0xffffffffu, (unsigned long long)t, src);
        const int64_t a = __shfl_sync(0xffffffffu, lo, src), b = __shfl_sync(0xffffffffu, hi, src);
        const uint32_t vv = __shfl_sync(0xffffffffu, v, src);
        for (int64_t c = a + lane; c < b; c += 32) tt[c] = vv;
    }
}

// cellT[c] = first sorted index whose dense-level cell is >= c, for
// c = 0 .. ncell (cellT[ncell] = n); position s writes the cells after its
// predecessor's up to its own.
__global__ void cell_table_kernel(const uint64_t *__restrict__ keys, int64_t n, int shift,
                                  int64_t ncell, uint32_t *__restrict__ cellT)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); s0 <= n; s0 += stride) {
        const int64_t s = s0 + (threadIdx.x & 31u);
        const bool act = s <= n;
        int64_t cs = 0, cp = 0;
        if (act) {
            cs = s < n ? (int64_t)(keys[s] >> shift) : ncell;
            cp = s > 0 ? (int64_t)(keys[s - 1] >> shift) : -1;
        }
        fill_runs(cellT, cp + 1, cs + 1, (uint32_t)s, act);
    }
}

// Batched pass: every subvolume's table at its own dense level, entries
// holding global sorted positions, from the keys that still carry the
// subvolume field.
__global__ void cell_table_seg_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                      const SegDesc *__restrict__ seg, uint32_t *__restrict__ cellT)
{
    const uint64_t m48 = (uint64_t(1) << 48) - 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); s0 < n; s0 += stride) {
        const int64_t s = s0 + (threadIdx.x & 31u);
        const bool act = s < n;
        uint32_t *t = cellT;
        int64_t cs = 0, cp = 0, ncell = 0;
        bool last = false;
        if (act) {
            const uint64_t key = keys[s];
            const SegDesc &d = seg[key >> 48];
            const int shift = 3 * (kMaxLevel - d.level_dense);
            ncell = int64_t(1) << (3 * d.level_dense);
            t = cellT + d.cell0;
            cs = (int64_t)((key & m48) >> shift);
            cp = s > d.base ? (int64_t)((keys[s - 1] & m48) >> shift) : -1;
            last = s == d.base + d.n - 1;
        }
        fill_runs(t, cp + 1, cs + 1, (uint32_t)s, act);
        fill_runs(t, cs + 1, ncell + 1, (uint32_t)(s + 1), last);
    }
}

// One warp per chunk of Q sorted particles: the chunk's level (cell side
// just >= its bounding-box extent) and the particle counts of the 3x3x3
// cells around the cell holding the box centre.  Writes, as requested:
//   feat[c][27] = log(1 + count), lvl[c], the closed-form radius
//   R = side * (81 k / (4 pi sum counts))^(1/3) * exp(log_margin)
//   (the radius of a ball holding k particles at the stencil's mean
//   density), and the training target log(max r_k over the chunk / side).
// With seg set (a batched pass) each chunk uses its subvolume's box, cell
// table and particle range.
template <typename T>
__global__ void chunk_feat_kernel(const typename V4<T>::type *__restrict__ spos,
                                  const uint64_t *__restrict__ keys,
                                  const uint32_t *__restrict__ cellT_all, int Ld_all, int64_t n_all,
                                  int64_t n_chunks, int Q, T box_all, T inv_box_all, int k,
                                  float log_margin, float *__restrict__ chunk_r,
                                  float *__restrict__ feat, uint8_t *__restrict__ lvl,
                                  const float *__restrict__ rk_s, float *__restrict__ target,
                                  const SegDesc *__restrict__ seg, int B)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ch = warp0; ch < n_chunks; ch += nwarps) {
        uint32_t cnt, tot;
        int l;
        double side;
        float rk;
        chunk_stencil<T>((const typename Vec4<T>::type *)spos, keys, cellT_all, Ld_all, n_all, Q, box_all,
                         inv_box_all, seg, B, ch, rk_s, lane, cnt, tot, l, side, rk);
        if (feat && lane < 27) feat[ch * HOP_MLP_IN + lane] = log1pf((float)cnt);
        if (lane == 0) {
            if (lvl) lvl[ch] = (uint8_t)l;
            if (chunk_r) {
                const double r = side * cbrt(81.0 * k / (4.0 * 3.14159265358979323846 * (double)max(tot, 1u)));
                chunk_r[ch] = (float)(r * exp((double)log_margin));
            }
            if (target) target[ch] = logf(fmaxf(rk, 1e-30f) / (float)side);
        }
    }
}

template <typename T>
int grid_build_t(hop_ctx *c, const T *pos, int64_t n, double box, void **spos_out,
                 uint32_t **perm_out, uint64_t **keys_out, uint32_t **cellT_out, int *Ld_out)
{
    uint64_t *k0 = (uint64_t *)ctx_buf(c, S_KEY0, n * sizeof(uint64_t));
    uint64_t *k1 = (uint64_t *)ctx_buf(c, S_KEY1, n * sizeof(uint64_t));
    uint32_t *v0 = (uint32_t *)ctx_buf(c, S_VAL0, n * sizeof(uint32_t));
    uint32_t *v1 = (uint32_t *)ctx_buf(c, S_VAL1, n * sizeof(uint32_t));
    void *tmp = ctx_buf(c, S_SORT_TMP, radix_sort_scratch_bytes(n));
    auto *spos = (typename V4<T>::type *)ctx_buf(c, S_SPOS, n * sizeof(typename V4<T>::type));
    const int Ld = dense_level_for(n);
    const int64_t ncell = int64_t(1) << (3 * Ld);
    uint32_t *cellT = (uint32_t *)ctx_buf(c, S_CELLT, (ncell + 1) * sizeof(uint32_t));
    if (!k0 || !k1 || !v0 || !v1 || !tmp || !spos || !cellT) return HOP_ENOMEM;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 32);
    if (blocks < 1) blocks = 1;
    keys_kernel<T><<<blocks, 256, 0, c->stream>>>(pos, n, (T)box, (T)(1.0 / box), k0, v0, c->d_err);
    HOP_LAUNCH(c);
    int rc = radix_sort_u64(c, k0, k1, v0, v1, n, 0, 48, tmp);
    if (rc) return rc;
    gather_kernel<T><<<blocks, 256, 0, c->stream>>>(pos, v0, n, spos, nullptr, nullptr);
    HOP_LAUNCH(c);
    int blocks2 = (int)std::min<int64_t>((n + 256) / 256, (int64_t)c->num_sms * 32);
    cell_table_kernel<<<blocks2, 256, 0, c->stream>>>(k0, n, 3 * (kMaxLevel - Ld), ncell, cellT);
    HOP_LAUNCH(c);
    *spos_out = spos;
    *perm_out = v0;
    *keys_out = k0;
    *cellT_out = cellT;
    *Ld_out = Ld;
    return HOP_OK;
}

template <typename T>
int chunk_feat_launch(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
                      int Ld, int64_t n, double box, int qpw, int k, float log_margin,
                      float *chunk_r, float *feat, uint8_t *lvl, const float *rk_s, float *target)
{
    const int64_t n_chunks = (n + qpw - 1) / qpw;
    int64_t blocks = (n_chunks + 7) / 8;
    blocks = std::min<int64_t>(blocks, (int64_t)c->num_sms * 16);
    if (blocks < 1) blocks = 1;
    chunk_feat_kernel<T><<<(unsigned)blocks, 256, 0, c->stream>>>(
        (const typename V4<T>::type *)spos, keys, cellT, Ld, n, n_chunks, qpw, (T)box,
        (T)(1.0 / box), k, log_margin, chunk_r, feat, lvl, rk_s, target, nullptr, 0);
    HOP_LAUNCH(c);
    return HOP_OK;
}

}  // namespace

int grid_build(hop_ctx *c, const void *pos, int64_t n, const hop_params *p, void **spos_out,
               uint32_t **perm_out, uint64_t **keys_out, uint32_t **cellT_out, int *Ld_out)
{
    if (p->pos_is_f64)
        return grid_build_t<double>(c, (const double *)pos, n, p->box, spos_out, perm_out,
                                    keys_out, cellT_out, Ld_out);
    return grid_build_t<float>(c, (const float *)pos, n, p->box, spos_out, perm_out, keys_out,
                               cellT_out, Ld_out);
}

// Closed-form first radius per chunk (HOP_RADIUS_COUNT), margin exp(0.25).
int chunk_radius(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
                 int Ld, int64_t n, const hop_params *p, int qpw, float *chunk_r)
{
    const float margin = 0.25f;
    if (p->pos_is_f64)
        return chunk_feat_launch<double>(c, spos, keys, cellT, Ld, n, p->box, qpw, p->n_dens,
                                         margin, chunk_r, nullptr, nullptr, nullptr, nullptr);
    return radius_closed(c, spos, keys, cellT, Ld, n, (n + qpw - 1) / qpw, qpw, p->box, nullptr, 0, p->n_dens, margin,
                         chunk_r);
}

// Features, levels and (if rk_s) targets for every chunk.
int chunk_features(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
                   int Ld, int64_t n, bool f64, double box, int qpw, float *feat, uint8_t *lvl,
                   const float *rk_s, float *target)
{
    if (f64)
        return chunk_feat_launch<double>(c, spos, keys, cellT, Ld, n, box, qpw, 64, 0.f, nullptr,
                                         feat, lvl, rk_s, target);
    return chunk_feat_launch<float>(c, spos, keys, cellT, Ld, n, box, qpw, 64, 0.f, nullptr, feat,
                                    lvl, rk_s, target);
}

// ------------------------------------------------------- batched pass ----
int grid_build_seg(hop_ctx *c, const float *pos, int64_t n, const SegDesc *seg, int B,
                   int64_t n_cells, void **spos_out, uint32_t **perm_out, uint64_t **keys_out,
                   uint32_t **cellT_out)
{
    uint64_t *k0 = (uint64_t *)ctx_buf(c, S_KEY0, n * sizeof(uint64_t));
    uint64_t *k1 = (uint64_t *)ctx_buf(c, S_KEY1, n * sizeof(uint64_t));
    uint32_t *v0 = (uint32_t *)ctx_buf(c, S_VAL0, n * sizeof(uint32_t));
    uint32_t *v1 = (uint32_t *)ctx_buf(c, S_VAL1, n * sizeof(uint32_t));
    void *tmp = ctx_buf(c, S_SORT_TMP, radix_sort_scratch_bytes(n));
    float4 *spos = (float4 *)ctx_buf(c, S_SPOS, n * sizeof(float4));
    uint32_t *cellT = (uint32_t *)ctx_buf(c, S_CELLT, n_cells * sizeof(uint32_t));
    if (!k0 || !k1 || !v0 || !v1 || !tmp || !spos || !cellT) return HOP_ENOMEM;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 32);
    if (blocks < 1) blocks = 1;
    keys_seg_kernel<float><<<blocks, 256, 0, c->stream>>>(pos, n, seg, B, k0, v0, c->d_err);
    HOP_LAUNCH(c);
    int sub_bits = 0;
    while ((1 << sub_bits) < B) sub_bits += 8;
    int rc = radix_sort_u64(c, k0, k1, v0, v1, n, 0, 48 + sub_bits, tmp);
    if (rc) return rc;
    // k0: sorted keys with the subvolume field; k1: the same without it
    gather_kernel<float><<<blocks, 256, 0, c->stream>>>(pos, v0, n, spos, k0, k1);
    HOP_LAUNCH(c);
    cell_table_seg_kernel<<<blocks, 256, 0, c->stream>>>(k0, n, seg, cellT);
    HOP_LAUNCH(c);
    *spos_out = spos;
    *perm_out = v0;
    *keys_out = k1;
    *cellT_out = cellT;
    return HOP_OK;
}

// Closed-form first radius of every chunk of a batched pass.
int chunk_radius_seg(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
                     const SegDesc *seg, int B, int64_t n_chunks, int qpw, int k, float *chunk_r)
{
    return radius_closed(c, spos, keys, cellT, 0, 0, n_chunks, qpw, 1.0, seg, B, k, 0.25f, chunk_r);
}
