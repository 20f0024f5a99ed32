// Learned first search radius: a 3-layer MLP (27 -> 64 -> 64 -> 1, ReLU)
// over log(1 + count) of a query chunk's 3x3x3 stencil cells, predicting
// log(largest Ndens-th-neighbour distance of the chunk / cell side).
// Weights are BF16 (an fp32 master copy is kept for training); products and
// sums are FP32.  Forward, backward and Adam are hand-written here.
#include "hop_internal.cuh"
#include "chunk_stencil.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

constexpr int IN = HOP_MLP_IN, H = HOP_MLP_HID, NP = HOP_MLP_NPARAM;
constexpr int oW1 = 0, oB1 = H * IN, oW2 = oB1 + H, oB2 = oW2 + H * H, oW3 = oB2 + H, oB3 = oW3 + H;
static_assert(oB3 + 1 == NP, "parameter layout");
constexpr int kGradThreads = 64;

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// Forward pass of one sample with weights W (fp32 values of the bf16 copy).
__device__ __forceinline__ float mlp_forward_one(const float *W, const float *x, float *h1)
{
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
        float a = W[oB1 + j];
#pragma unroll
        for (int f = 0; f < IN; ++f) a = fmaf(W[oW1 + j * IN + f], x[f], a);
        h1[j] = fmaxf(a, 0.f);
    }
    float y = W[oB3];
    for (int o = 0; o < H; ++o) {
        float a = W[oB2 + o];
#pragma unroll
        for (int i = 0; i < H; ++i) a = fmaf(W[oW2 + o * H + i], h1[i], a);
        y = fmaf(W[oW3 + o], fmaxf(a, 0.f), y);
    }
    return y;
}

// out[s] = MLP(feat[s]); with lvl != null the output is the search radius
// side(lvl) * exp(y + margin) instead.
__global__ void mlp_fwd_kernel(const __nv_bfloat16 *__restrict__ w16, const float *__restrict__ feat,
                               int64_t m, float *__restrict__ out, const uint8_t *__restrict__ lvl,
                               double box, float margin)
{
    __shared__ float W[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) W[i] = bf(w16, i);
    __syncthreads();
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m;
         s += (int64_t)gridDim.x * blockDim.x) {
        float x[IN], h1[H];
#pragma unroll
        for (int f = 0; f < IN; ++f) x[f] = feat[s * IN + f];
        const float y = mlp_forward_one(W, x, h1);
        if (lvl) {
            const float sd = (float)(box / (double)(1u << lvl[s]));
            out[s] = sd * expf(y + margin);
        } else {
            out[s] = y;
        }
    }
}

// The first radius of every chunk in one pass, 32 chunks per warp: each
// lane finds its chunk's stencil level and centre cell (the same arithmetic
// as chunk_stencil), the warp looks up the 27 stencil cells of one chunk at
// a time (27 lanes), and each lane turns its chunk's counts into a radius.
// NET: the learned radius, R = side * exp(MLP + margin), the network run
// with its activations in registers.  !NET: the closed form from the
// stencil total, R = side * cbrt(81 k / (4 pi total)) * exp(margin), the
// chunk's k-th-neighbour distance if the 27 cells held the mean density of
// their total.
// Weights sit in shared memory as fp32 values of the bf16 copy, laid out
// so that a lane reads four consecutive outputs' weights at once.
constexpr int kRadThreads = 128;
constexpr int kRadWarps = kRadThreads / 32;
constexpr int kFeatStride = IN + 2;   // 29: lane-strided feature rows hit distinct banks
static_assert(H % 16 == 0, "hidden width in blocks of 16");

struct RadWeights {
    float w1t[IN][H];   // w1t[f][j] = W1[j][f]
    float b1[H];
    float w2t[H][H];    // w2t[i][o] = W2[o][i]
    float b2[H];
    float w3[H];
    float b3;
};

template <bool NET>
__global__ void __launch_bounds__(kRadThreads, 4)
radius_kernel(const __nv_bfloat16 *__restrict__ w16, const float4 *__restrict__ spos,
              const uint64_t *__restrict__ keys, const uint32_t *__restrict__ cellT, int Ld,
              int64_t n, int64_t n_chunks, int Q, float box, float inv_box,
              const SegDesc *__restrict__ seg, int B, float margin, int k, float *__restrict__ chunk_r)
{
    __shared__ __align__(16) RadWeights Ws;
    __shared__ float F[kRadWarps][32][kFeatStride];
    __shared__ uint32_t T[kRadWarps][32];
    if constexpr (NET) {
        for (int i = threadIdx.x; i < H * IN; i += blockDim.x) Ws.w1t[i % IN][i / IN] = bf(w16, oW1 + i);
        for (int i = threadIdx.x; i < H * H; i += blockDim.x) Ws.w2t[i % H][i / H] = bf(w16, oW2 + i);
        for (int i = threadIdx.x; i < H; i += blockDim.x) {
            Ws.b1[i] = bf(w16, oB1 + i);
            Ws.b2[i] = bf(w16, oB2 + i);
            Ws.w3[i] = bf(w16, oW3 + i);
        }
        if (threadIdx.x == 0) Ws.b3 = bf(w16, oB3);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * kRadWarps * 32;
    for (int64_t base = ((int64_t)blockIdx.x * kRadWarps + w) * 32; base < n_chunks; base += stride) {
        const int nc = (int)min((int64_t)32, n_chunks - base);
        // ---- the lane's chunk: stencil level, centre cell, cell side
        const int64_t ch = base + (lane < nc ? lane : 0);
        int64_t s0 = ch * Q, nend = n, cell0 = 0;
        int ld = Ld;
        float bx = box, ibx = inv_box;
        if (seg) {
            const SegDesc &d = seg[seg_of_chunk(seg, B, ch)];
            s0 = d.base + (ch - d.chunk0) * Q;
            nend = d.base + d.n;
            cell0 = d.cell0;
            ld = d.level_dense;
            bx = (float)d.box;
            ibx = (float)(1.0 / d.box);
        }
        const int nq = (int)min((int64_t)Q, nend - s0);
        float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
        for (int q = 0; q < nq; ++q) {
            const float4 v = spos[s0 + q];
            lx = fminf(lx, v.x);
            ly = fminf(ly, v.y);
            lz = fminf(lz, v.z);
            hx = fmaxf(hx, v.x);
            hy = fmaxf(hy, v.y);
            hz = fmaxf(hz, v.z);
        }
        const float ext = fmaxf(hx - lx, fmaxf(hy - ly, hz - lz));
        int l = kMaxLevel;
        while (l > 2 && bx / (float)(1 << l) < ext) --l;
        const int G = 1 << l;
        const float sc = ibx * (float)G;
        const int cx = min((int)floorf((lx + hx) * 0.5f * sc), G - 1);
        const int cy = min((int)floorf((ly + hy) * 0.5f * sc), G - 1);
        const int cz = min((int)floorf((lz + hz) * 0.5f * sc), G - 1);
        const float side = (float)((double)bx / (double)G);
        // ---- the 27 stencil counts of each chunk, one chunk at a time
        const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
        for (int j = 0; j < nc; ++j) {
            const int lj = __shfl_sync(0xffffffffu, l, j), ldj = __shfl_sync(0xffffffffu, ld, j);
            const int xj = __shfl_sync(0xffffffffu, cx, j), yj = __shfl_sync(0xffffffffu, cy, j),
                      zj = __shfl_sync(0xffffffffu, cz, j);
            const int64_t c0 = __shfl_sync(0xffffffffu, cell0, j);
            uint32_t cnt = 0;
            if (lane < IN) {
                const int Gj = 1 << lj;
                const int rx = (xj + dx + Gj) % Gj, ry = (yj + dy + Gj) % Gj, rz = (zj + dz + Gj) % Gj;
                uint32_t a, b;
                cell_range(cellT + c0, keys, ldj, lj, morton3((uint32_t)rx, (uint32_t)ry, (uint32_t)rz), a, b);
                cnt = b - a;
                if constexpr (NET) F[w][j][lane] = log1pf((float)cnt);
            }
            if constexpr (!NET) {
                const uint32_t tot = __reduce_add_sync(0xffffffffu, cnt);
                if (lane == 0) T[w][j] = tot;
            }
        }
        __syncwarp();
        if constexpr (!NET) {
            if (lane < nc) {
                const double r = (double)side * cbrt(81.0 * k / (4.0 * 3.14159265358979323846 * (double)max(T[w][lane], 1u)));
                chunk_r[base + lane] = (float)(r * exp((double)margin));
            }
            __syncwarp();
            continue;
        }
        // ---- the network for the lane's chunk
        if (lane < nc) {
            const float *x = F[w][lane];
            float h[H];
#pragma unroll
            for (int j = 0; j < H; ++j) h[j] = Ws.b1[j];
            for (int f = 0; f < IN; ++f) {
                const float xf = x[f];
                const float4 *r = (const float4 *)Ws.w1t[f];
#pragma unroll
                for (int j4 = 0; j4 < H / 4; ++j4) {
                    const float4 wv = r[j4];
                    h[4 * j4 + 0] = fmaf(wv.x, xf, h[4 * j4 + 0]);
                    h[4 * j4 + 1] = fmaf(wv.y, xf, h[4 * j4 + 1]);
                    h[4 * j4 + 2] = fmaf(wv.z, xf, h[4 * j4 + 2]);
                    h[4 * j4 + 3] = fmaf(wv.w, xf, h[4 * j4 + 3]);
                }
            }
#pragma unroll
            for (int j = 0; j < H; ++j) h[j] = fmaxf(h[j], 0.f);
            float y = Ws.b3;
            for (int ob = 0; ob < H; ob += 16) {
                float acc[16];
#pragma unroll
                for (int m = 0; m < 16; ++m) acc[m] = Ws.b2[ob + m];
#pragma unroll
                for (int i = 0; i < H; ++i) {
                    const float4 *r = (const float4 *)&Ws.w2t[i][ob];
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const float4 wv = r[k4];
                        acc[4 * k4 + 0] = fmaf(wv.x, h[i], acc[4 * k4 + 0]);
                        acc[4 * k4 + 1] = fmaf(wv.y, h[i], acc[4 * k4 + 1]);
                        acc[4 * k4 + 2] = fmaf(wv.z, h[i], acc[4 * k4 + 2]);
                        acc[4 * k4 + 3] = fmaf(wv.w, h[i], acc[4 * k4 + 3]);
                    }
                }
#pragma unroll
                for (int m = 0; m < 16; ++m) y = fmaf(Ws.w3[ob + m], fmaxf(acc[m], 0.f), y);
            }
            chunk_r[base + lane] = side * expf(y + margin);
        }
        __syncwarp();
    }
}

// Mean-squared-error gradient over a set of samples (idx[] or 0..m-1),
// scaled by `scale` (1 / batch size).  Each block keeps its samples'
// activations and back-propagated errors in shared memory and forms its share
// of every parameter gradient as a sum over those samples, then adds it to
// the global gradient.
__global__ void mlp_grad_kernel(const __nv_bfloat16 *__restrict__ w16, const float *__restrict__ feat,
                                const float *__restrict__ target, const uint32_t *__restrict__ idx,
                                int64_t m, float scale, float *__restrict__ grad,
                                double *__restrict__ loss)
{
    extern __shared__ float sm[];
    float *W = sm;                    // NP
    float *G = W + NP;                // NP
    float *X = G + NP;                // T x IN
    float *H1 = X + kGradThreads * IN;   // T x H
    float *H2 = H1 + kGradThreads * H;   // T x H
    float *D2 = H2 + kGradThreads * H;   // T x H  (d loss / d pre-activation 2)
    float *D1 = D2 + kGradThreads * H;   // T x H  (d loss / d pre-activation 1)
    float *DY = D1 + kGradThreads * H;   // T
    const int t = threadIdx.x;
    for (int i = t; i < NP; i += blockDim.x) { W[i] = bf(w16, i); G[i] = 0.f; }
    __syncthreads();
    double lsum = 0.0;
    for (int64_t base = (int64_t)blockIdx.x * kGradThreads; base < m;
         base += (int64_t)gridDim.x * kGradThreads) {
        const int64_t sidx = base + t;
        const bool valid = sidx < m;
        const int64_t s = valid ? (idx ? (int64_t)idx[sidx] : sidx) : 0;
        float *x = X + t * IN, *h1 = H1 + t * H, *h2 = H2 + t * H, *d2 = D2 + t * H, *d1 = D1 + t * H;
        for (int f = 0; f < IN; ++f) x[f] = valid ? feat[s * IN + f] : 0.f;
        for (int j = 0; j < H; ++j) {
            float a = W[oB1 + j];
            for (int f = 0; f < IN; ++f) a = fmaf(W[oW1 + j * IN + f], x[f], a);
            h1[j] = fmaxf(a, 0.f);
        }
        float y = W[oB3];
        for (int o = 0; o < H; ++o) {
            float a = W[oB2 + o];
            for (int i = 0; i < H; ++i) a = fmaf(W[oW2 + o * H + i], h1[i], a);
            h2[o] = fmaxf(a, 0.f);
            y = fmaf(W[oW3 + o], h2[o], y);
        }
        const float r = valid ? y - target[s] : 0.f;
        lsum += (double)r * (double)r * (double)scale;
        const float dy = 2.f * r * scale;
        DY[t] = dy;
        for (int o = 0; o < H; ++o) d2[o] = h2[o] > 0.f ? dy * W[oW3 + o] : 0.f;
        for (int i = 0; i < H; ++i) {
            float a = 0.f;
            for (int o = 0; o < H; ++o) a = fmaf(W[oW2 + o * H + i], d2[o], a);
            d1[i] = h1[i] > 0.f ? a : 0.f;
        }
        __syncthreads();
        for (int pidx = t; pidx < NP; pidx += blockDim.x) {
            float acc = 0.f;
            if (pidx < oB1) {
                const int j = pidx / IN, f = pidx % IN;
                for (int u = 0; u < kGradThreads; ++u) acc = fmaf(D1[u * H + j], X[u * IN + f], acc);
            } else if (pidx < oW2) {
                const int j = pidx - oB1;
                for (int u = 0; u < kGradThreads; ++u) acc += D1[u * H + j];
            } else if (pidx < oB2) {
                const int o = (pidx - oW2) / H, i = (pidx - oW2) % H;
                for (int u = 0; u < kGradThreads; ++u) acc = fmaf(D2[u * H + o], H1[u * H + i], acc);
            } else if (pidx < oW3) {
                const int o = pidx - oB2;
                for (int u = 0; u < kGradThreads; ++u) acc += D2[u * H + o];
            } else if (pidx < oB3) {
                const int o = pidx - oW3;
                for (int u = 0; u < kGradThreads; ++u) acc = fmaf(DY[u], H2[u * H + o], acc);
            } else {
                for (int u = 0; u < kGradThreads; ++u) acc += DY[u];
            }
            G[pidx] += acc;
        }
        __syncthreads();
    }
    for (int i = t; i < NP; i += blockDim.x) atomicAdd(&grad[i], G[i]);
    // block-reduce the loss
    __shared__ double lred[kGradThreads];
    lred[t] = lsum;
    __syncthreads();
    if (t == 0) {
        double a = 0.0;
        for (int u = 0; u < kGradThreads; ++u) a += lred[u];
        atomicAdd(loss, a);
    }
}

__global__ void adam_kernel(float *__restrict__ w, __nv_bfloat16 *__restrict__ w16,
                            float *__restrict__ mo, float *__restrict__ ve,
                            const float *__restrict__ g, float lr, float bc1, float bc2)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NP; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float m = b1 * mo[i] + (1.f - b1) * gi;
        const float v = b2 * ve[i] + (1.f - b2) * gi * gi;
        mo[i] = m;
        ve[i] = v;
        const float mh = m / bc1, vh = v / bc2;
        const float nw = w[i] - lr * mh / (sqrtf(vh) + eps);
        w[i] = nw;
        w16[i] = __float2bfloat16_rn(nw);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ w16, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w16[i] = __float2bfloat16_rn(w[i]);
}

size_t grad_smem_bytes()
{
    return sizeof(float) * (2 * NP + kGradThreads * IN + 4 * kGradThreads * H + kGradThreads);
}

int grad_launch(hop_ctx *c, const float *feat, const float *target, const uint32_t *idx, int64_t m,
                float scale, float *grad, double *loss)
{
    const size_t smem = grad_smem_bytes();
    HOP_CUDA(c, cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t blocks = (m + kGradThreads - 1) / kGradThreads;
    blocks = std::min<int64_t>(blocks, (int64_t)c->num_sms * 2);
    blocks = std::max<int64_t>(blocks, 1);
    mlp_grad_kernel<<<(unsigned)blocks, kGradThreads, smem, c->stream>>>(
        (const __nv_bfloat16 *)c->mlp->w16, feat, target, idx, m, scale, grad, loss);
    HOP_LAUNCH(c);
    return HOP_OK;
}

}  // namespace

int mlp_ensure(hop_ctx *c)
{
    if (c->mlp->w32) return HOP_OK;
    char *p = nullptr;
    const size_t bytes = sizeof(float) * NP * 4 + sizeof(uint16_t) * NP + 256;
    HOP_CUDA(c, cudaMalloc(&p, bytes));
    HOP_CUDA(c, cudaMemset(p, 0, bytes));
    c->mlp->w32 = (float *)p;
    c->mlp->m = c->mlp->w32 + NP;
    c->mlp->v = c->mlp->m + NP;
    c->mlp->g = c->mlp->v + NP;
    c->mlp->w16 = (uint16_t *)(c->mlp->g + NP);
    return HOP_OK;
}

void mlp_free(hop_ctx *c)
{
    for (MlpState &m : c->mlp_bank) {
        if (m.w32) cudaFree(m.w32);
        m = MlpState();
    }
}

int mlp_forward_dev(hop_ctx *c, const float *feat, int64_t m, float *out)
{
    int64_t blocks = std::min<int64_t>((m + 127) / 128, (int64_t)c->num_sms * 8);
    blocks = std::max<int64_t>(blocks, 1);
    mlp_fwd_kernel<<<(unsigned)blocks, 128, 0, c->stream>>>((const __nv_bfloat16 *)c->mlp->w16, feat, m,
                                                           out, nullptr, 1.0, 0.f);
    HOP_LAUNCH(c);
    return HOP_OK;
}

namespace {

int radius_fused(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT, int Ld,
                 int64_t n, int64_t n_chunks, int qpw, double box, const SegDesc *seg, int B, float *chunk_r)
{
    int64_t blocks = (n_chunks + kRadThreads - 1) / kRadThreads;
    blocks = std::min<int64_t>(blocks, (int64_t)c->num_sms * 4);
    blocks = std::max<int64_t>(blocks, 1);
    radius_kernel<true><<<(unsigned)blocks, kRadThreads, 0, c->stream>>>(
        (const __nv_bfloat16 *)c->mlp->w16, (const float4 *)spos, keys, cellT, Ld, n, n_chunks, qpw,
        (float)box, (float)(1.0 / box), seg, B, c->mlp->log_margin, 0, chunk_r);
    HOP_LAUNCH(c);
    return HOP_OK;
}

}  // namespace

// The closed-form radius (float32 positions) with the same kernel.
int radius_closed(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT, int Ld, int64_t n,
                  int64_t n_chunks, int qpw, double box, const SegDesc *seg, int B, int k, float log_margin,
                  float *chunk_r)
{
    int64_t blocks = (n_chunks + kRadThreads - 1) / kRadThreads;
    blocks = std::min<int64_t>(blocks, (int64_t)c->num_sms * 4);
    blocks = std::max<int64_t>(blocks, 1);
    radius_kernel<false><<<(unsigned)blocks, kRadThreads, 0, c->stream>>>(
        nullptr, (const float4 *)spos, keys, cellT, Ld, n, n_chunks, qpw, (float)box, (float)(1.0 / box), seg, B,
        log_margin, k, chunk_r);
    HOP_LAUNCH(c);
    return HOP_OK;
}

int mlp_radius(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT, int Ld,
               int64_t n, const hop_params *p, int qpw, float *chunk_r)
{
    const int64_t nc = (n + qpw - 1) / qpw;
    if (!p->pos_is_f64) return radius_fused(c, spos, keys, cellT, Ld, n, nc, qpw, p->box, nullptr, 0, chunk_r);
    float *feat = (float *)ctx_buf(c, S_MLP_TMP, nc * IN * sizeof(float));
    uint8_t *lvl = (uint8_t *)ctx_buf(c, S_CHUNK_LVL, nc);
    if (!feat || !lvl) return HOP_ENOMEM;
    int rc = chunk_features(c, spos, keys, cellT, Ld, n, p->pos_is_f64 != 0, p->box, qpw, feat, lvl,
                            nullptr, nullptr);
    if (rc) return rc;
    int64_t blocks = std::min<int64_t>((nc + 127) / 128, (int64_t)c->num_sms * 8);
    blocks = std::max<int64_t>(blocks, 1);
    mlp_fwd_kernel<<<(unsigned)blocks, 128, 0, c->stream>>>((const __nv_bfloat16 *)c->mlp->w16, feat, nc,
                                                           chunk_r, lvl, p->box, c->mlp->log_margin);
    HOP_LAUNCH(c);
    return HOP_OK;
}

// Batched pass: features of every chunk (with the cell side of its own
// subvolume in chunk_r), then radius = side * exp(MLP + margin) in place.
int mlp_radius_seg(hop_ctx *c, const void *spos, const uint64_t *keys, const uint32_t *cellT,
                   const SegDesc *seg, int B, int64_t n_chunks, int qpw, int k, float *chunk_r)
{
    if (!c->mlp->loaded) return ctx_fail(c, HOP_ENOMODEL, "no radius network loaded (hop_mlp_load)");
    (void)k;
    return radius_fused(c, spos, keys, cellT, 0, 0, n_chunks, qpw, 1.0, seg, B, chunk_r);
}

extern "C" {

int hop_mlp_load(hop_ctx *c, const float *params_host, float log_margin)
{
    if (!c || !params_host) return HOP_EINVAL;
    HOP_CUDA(c, cudaSetDevice(c->device));
    int rc = mlp_ensure(c);
    if (rc) return rc;
    HOP_CUDA(c, cudaMemcpyAsync(c->mlp->w32, params_host, sizeof(float) * NP, cudaMemcpyHostToDevice, c->stream));
    HOP_CUDA(c, cudaMemsetAsync(c->mlp->m, 0, sizeof(float) * NP * 2, c->stream));
    to_bf16_kernel<<<8, 256, 0, c->stream>>>(c->mlp->w32, (__nv_bfloat16 *)c->mlp->w16, NP);
    HOP_LAUNCH(c);
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    c->mlp->loaded = true;
    c->mlp->log_margin = log_margin;
    c->mlp->step = 0;
    return HOP_OK;
}

int hop_mlp_get(hop_ctx *c, float *params_host)
{
    if (!c || !params_host) return HOP_EINVAL;
    if (!c->mlp->loaded) return ctx_fail(c, HOP_ENOMODEL, "no network loaded");
    HOP_CUDA(c, cudaMemcpyAsync(params_host, c->mlp->w32, sizeof(float) * NP, cudaMemcpyDeviceToHost, c->stream));
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    return HOP_OK;
}

int hop_mlp_samples(hop_ctx *c, float *feat, float *target, int64_t cap, int64_t *n_chunks)
{
    if (!c || !n_chunks) return HOP_EINVAL;
    if (!c->last_spos) return ctx_fail(c, HOP_EINVAL, "no density pass to take samples from");
    const int64_t nc = (c->last_n + c->last_qpw - 1) / c->last_qpw;
    *n_chunks = nc;
    if (!feat || !target) return HOP_OK;
    if (cap < nc) return ctx_fail(c, HOP_ETABLE, "sample capacity too small");
    HOP_CUDA(c, cudaSetDevice(c->device));
    uint8_t *lvl = (uint8_t *)ctx_buf(c, S_CHUNK_LVL, nc);
    if (!lvl) return HOP_ENOMEM;
    int rc = chunk_features(c, c->last_spos, c->last_keys, c->last_cellT, c->last_level_dense, c->last_n,
                            c->last_f64, c->last_box, c->last_qpw, feat, lvl, c->last_rk, target);
    if (rc) return rc;
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    return HOP_OK;
}

int hop_mlp_forward(hop_ctx *c, const float *feat, int64_t m, float *out)
{
    if (!c || !feat || !out || m < 0) return HOP_EINVAL;
    if (!c->mlp->loaded) return ctx_fail(c, HOP_ENOMODEL, "no network loaded");
    HOP_CUDA(c, cudaSetDevice(c->device));
    if (m == 0) return HOP_OK;
    return mlp_forward_dev(c, feat, m, out);
}

int hop_mlp_grad(hop_ctx *c, const float *feat, const float *target, int64_t m, double *loss,
                 float *grad)
{
    if (!c || !feat || !target || !grad || !loss || m <= 0) return HOP_EINVAL;
    if (!c->mlp->loaded) return ctx_fail(c, HOP_ENOMODEL, "no network loaded");
    HOP_CUDA(c, cudaSetDevice(c->device));
    double *dl = (double *)ctx_buf(c, S_MISC, 256);
    if (!dl) return HOP_ENOMEM;
    HOP_CUDA(c, cudaMemsetAsync(grad, 0, sizeof(float) * NP, c->stream));
    HOP_CUDA(c, cudaMemsetAsync(dl, 0, sizeof(double), c->stream));
    int rc = grad_launch(c, feat, target, nullptr, m, 1.f / (float)m, grad, dl);
    if (rc) return rc;
    HOP_CUDA(c, cudaMemcpyAsync(c->h_pinned, dl, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HOP_CUDA(c, cudaStreamSynchronize(c->stream));
    *loss = *(double *)c->h_pinned;
    return HOP_OK;
}

int hop_mlp_train(hop_ctx *c, const float *feat, const float *target, int64_t m, int32_t epochs,
                  int32_t batch, float lr, uint64_t seed, double *final_loss)
{
    if (!c || !feat || !target || m <= 0 || epochs <= 0 || batch <= 0) return HOP_EINVAL;
    if (!c->mlp->loaded) return ctx_fail(c, HOP_ENOMODEL, "load initial parameters first (hop_mlp_load)");
    HOP_CUDA(c, cudaSetDevice(c->device));
    uint32_t *perm = (uint32_t *)ctx_buf(c, S_MLP_TMP, m * sizeof(uint32_t));
    double *dl = (double *)ctx_buf(c, S_MISC, 256);
    if (!perm || !dl) return HOP_ENOMEM;
    std::vector<uint32_t> hp((size_t)m);
    uint64_t st = seed;
    auto next = [&]() {
        // SplitMix64 step (Steele, Lea & Flood 2014)
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < m; ++i) hp[i] = (uint32_t)i;
        for (int64_t i = m - 1; i > 0; --i) std::swap(hp[i], hp[next() % (uint64_t)(i + 1)]);
        HOP_CUDA(c, cudaMemcpyAsync(perm, hp.data(), m * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
        HOP_CUDA(c, cudaMemsetAsync(dl, 0, sizeof(double), c->stream));
        for (int64_t b = 0; b < m; b += batch) {
            const int64_t bs = std::min<int64_t>(batch, m - b);
            HOP_CUDA(c, cudaMemsetAsync(c->mlp->g, 0, sizeof(float) * NP, c->stream));
            // loss of each batch is its mean; weight it by bs/m for the epoch mean
            int rc = grad_launch(c, feat, target, perm + b, bs, 1.f / (float)bs, c->mlp->g, dl);
            if (rc) return rc;
            c->mlp->step += 1;
            const float bc1 = 1.f - powf(0.9f, (float)c->mlp->step);
            const float bc2 = 1.f - powf(0.999f, (float)c->mlp->step);
            adam_kernel<<<(NP + 255) / 256, 256, 0, c->stream>>>(c->mlp->w32, (__nv_bfloat16 *)c->mlp->w16,
                                                                c->mlp->m, c->mlp->v, c->mlp->g, lr, bc1, bc2);
            HOP_LAUNCH(c);
        }
        HOP_CUDA(c, cudaMemcpyAsync(c->h_pinned, dl, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        HOP_CUDA(c, cudaStreamSynchronize(c->stream));
        // sum over batches of (batch mean loss); convert to a per-sample mean
        const double nb = (double)((m + batch - 1) / batch);
        last = *(double *)c->h_pinned / nb;
    }
    if (final_loss) *final_loss = last;
    return HOP_OK;
}

}  // extern "C"
