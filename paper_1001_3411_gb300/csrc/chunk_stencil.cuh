// The 3x3x3 stencil of a query chunk, shared by the feature kernel
// (grid.cu: features, closed-form radii, training targets) and the fused
// feature + network radius kernel (mlp.cu).
#pragma once

#include "hop_internal.cuh"
#include "knn_common.cuh"

namespace {

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4; };

// One warp, one chunk of Q <= 32 consecutive sorted particles (lane j holds
// particle j).  The chunk's level is the finest whose cell side covers the
// chunk's bounding-box extent; the stencil is the 3x3x3 cells of that level
// around the cell holding the box centre.  Lane j < 27 gets the particle
// count of stencil cell j; every lane gets the stencil total, the level,
// the cell side and (if rk_s) the largest r_k of the chunk.  With seg set
// the chunk belongs to its subvolume (box, cell table, particle range).
template <typename T>
__device__ __forceinline__ void chunk_stencil(const typename Vec4<T>::type *__restrict__ spos,
                                              const uint64_t *__restrict__ keys,
                                              const uint32_t *__restrict__ cellT_all, int Ld_all,
                                              int64_t n_all, int Q, T box_all, T inv_box_all,
                                              const SegDesc *__restrict__ seg, int B, int64_t ch,
                                              const float *__restrict__ rk_s, int lane, uint32_t &cnt,
                                              uint32_t &tot, int &level, double &side, float &rk)
{
    int64_t s0 = ch * Q, n = n_all;
    const uint32_t *cellT = cellT_all;
    int Ld = Ld_all;
    T box = box_all, inv_box = inv_box_all;
    if (seg) {
        const SegDesc &d = seg[seg_of_chunk(seg, B, ch)];
        s0 = d.base + (ch - d.chunk0) * Q;
        n = d.base + d.n;
        cellT = cellT_all + d.cell0;
        Ld = d.level_dense;
        box = (T)d.box;
        inv_box = (T)(1.0 / d.box);
    }
    const int nq = (int)min((int64_t)Q, n - s0);
    const int64_t s = s0 + (lane < nq ? lane : 0);
    const typename Vec4<T>::type v = spos[s];
    T lx = v.x, ly = v.y, lz = v.z, hx = v.x, hy = v.y, hz = v.z;
    rk = (rk_s && lane < nq) ? rk_s[s] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = min(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = min(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = min(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = max(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = max(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = max(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        rk = fmaxf(rk, __shfl_xor_sync(0xffffffffu, rk, o));
    }
    const T ext = max(hx - lx, max(hy - ly, hz - lz));
    int l = kMaxLevel;
    while (l > 2 && box / (T)(1 << l) < ext) --l;
    const int G = 1 << l;
    const T sc = inv_box * (T)G;
    const int cx = min((int)floor((lx + hx) * T(0.5) * sc), G - 1);
    const int cy = min((int)floor((ly + hy) * T(0.5) * sc), G - 1);
    const int cz = min((int)floor((lz + hz) * T(0.5) * sc), G - 1);
    cnt = 0;
    if (lane < 27) {
        const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
        const int rx = (cx + dx + G) % G, ry = (cy + dy + G) % G, rz = (cz + dz + G) % G;
        uint32_t a, b;
        cell_range(cellT, keys, Ld, l, morton3((uint32_t)rx, (uint32_t)ry, (uint32_t)rz), a, b);
        cnt = b - a;
    }
    tot = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    level = l;
    side = (double)box / (double)G;
}

}  // namespace
