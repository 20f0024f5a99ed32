// Halo statistics: once the halos are known, Parallel HOP computes for
// each its dark matter mass, centre of mass and maximum radius (Sec. 3,
// end of the merging description).  Particle masses are equal, so the mass
// is the member count.  In the periodic box the centre of mass is taken
// about the halo's peak particle (its densest member, then the smaller
// index): members' minimum-image offsets from the peak are averaged and
// added to the peak's position, wrapped into [0, box).
//
// Arithmetic.  Coordinates are taken in fixed point, X = rn(x 2^32 / box)
// (int64, within 0.5 + 2^-12 units of the exact value), so the box is
// 2^32 units and minimum images are integer wraps.  The centre is the
// peak's X plus the mean of the members' wrapped offsets from it -- the
// mean of the members' unwrapped X, within 0.5 units of the exact centre
// whatever the order of the sums.  The maximum radius is the largest
// member distance from the centre rounded to units, its square summed
// exactly in uint64: within 1.5 units of the exact distance.  No per-member
// arithmetic runs in fp64 (GB300's fp64 rate is a small fraction of its
// fp32 rate); the split scale makes the fp32 product exact enough.
//
// Three passes over the particles, each HBM-bound: peak keys and counts,
// offset sums, then the radii; between them, per group, the peak's
// coordinates and the centre.  A warp reduces each run of consecutive lanes
// holding the same group with a segmented shuffle scan (five steps) and
// carries its last run on to the next 32 particles, so a halo's members,
// mostly consecutive in the input, cost few atomics.
#include "hop_internal.cuh"

#include <algorithm>

namespace {

constexpr long long kUnits = 1ll << 32;   // the box in fixed-point units

// rn(x * scale) for x in [0, box): the scale is split into two floats
// (hi + lo); x hi is exact as p + e (fmaf), and e + x lo is small, so one
// more rounding of the fractional part gives the integer.
__device__ __forceinline__ long long fixed_of(float x, float s_hi, float s_lo)
{
    const float p = x * s_hi;
    const float e = fmaf(x, s_hi, -p);
    const float t = fmaf(x, s_lo, e);
    const float pi = rintf(p);
    return (long long)pi + (long long)rintf((p - pi) + t);
}

__device__ __forceinline__ long long fixed_of(double x, float, float, double s) { return __double2ll_rn(x * s); }
__device__ __forceinline__ long long fixed_of(float x, float s_hi, float s_lo, double)
{
    return fixed_of(x, s_hi, s_lo);
}

__device__ __forceinline__ long long wrap_units(long long d)
{
    if (d > kUnits / 2) return d - kUnits;
    if (d < -kUnits / 2) return d + kUnits;
    return d;
}

struct Scale {
    double s;          // 2^32 / box
    float hi, lo;      // s split into two floats
};

// Each pass gives every warp spans of kHaloSpan consecutive particles, 32
// per step, loading kHaloU steps before reducing any of them.  Runs of equal
// group ids are reduced across the warp; every complete run goes to memory
// with one atomic, and the warp's last run is carried into the next step
// (members of a halo are mostly consecutive, so a large halo costs one
// atomic per span rather than one per step).
constexpr int kHaloU = 4;
constexpr int kHaloSteps = 32;
constexpr int kHaloSpan = 32 * kHaloSteps;

struct WarpSpan {
    int64_t w, nw;
    __device__ WarpSpan()
    {
        w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    }
};

__device__ __forceinline__ int last_head(uint32_t heads) { return 31 - __clz(heads); }

__global__ void halo_peak_kernel(const float *__restrict__ dens, const int32_t *__restrict__ group, int64_t n,
                                 int64_t G, unsigned long long *__restrict__ pkey,
                                 unsigned long long *__restrict__ count, uint32_t *__restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const WarpSpan ws;
    for (int64_t w0 = ws.w * kHaloSpan; w0 < n; w0 += ws.nw * kHaloSpan) {
        int32_t cg = -1;                      // the carried run: group, best key, length
        unsigned long long cbest = 0, ccnt = 0;
        for (int t = 0; t < kHaloSteps; t += kHaloU) {
            int32_t g[kHaloU];
            float dv[kHaloU];
#pragma unroll
            for (int u = 0; u < kHaloU; ++u) {
                const int64_t i = w0 + (int64_t)(t + u) * 32 + lane;
                g[u] = i < n ? group[i] : -1;
                dv[u] = i < n ? dens[i] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kHaloU; ++u) {
                const int64_t i = w0 + (int64_t)(t + u) * 32 + lane;
                int32_t gg = g[u];
                if (gg >= G) {
                    atomicOr(err, kErrBadIndex);
                    gg = -1;
                }
                if (!__any_sync(0xffffffffu, gg >= 0)) continue;
                const uint32_t heads = run_heads((int64_t)gg, lane);
                const unsigned long long key =
                    gg >= 0 ? ((unsigned long long)__float_as_uint(dv[u]) << 32) |
                                  (unsigned long long)(0xFFFFFFFFu - (uint32_t)i)
                            : 0ull;
                unsigned long long best = run_max(heads, lane, key);
                unsigned long long len = (unsigned long long)run_len(heads, lane);
                if (lane == 0 && cg >= 0) {
                    if (gg == cg) {
                        best = best > cbest ? best : cbest;
                        len += ccnt;
                    } else {
                        atomicMax(&pkey[cg], cbest);
                        atomicAdd(&count[cg], ccnt);
                    }
                }
                const int last = last_head(heads);
                if (gg >= 0 && ((heads >> lane) & 1u) && lane != last) {
                    atomicMax(&pkey[gg], best);
                    atomicAdd(&count[gg], len);
                }
                cg = __shfl_sync(0xffffffffu, gg, last);
                cbest = __shfl_sync(0xffffffffu, best, last);
                ccnt = __shfl_sync(0xffffffffu, len, last);
            }
        }
        if (lane == 0 && cg >= 0) {
            atomicMax(&pkey[cg], cbest);
            atomicAdd(&count[cg], ccnt);
        }
    }
}

// Per group: the peak's fixed-point coordinates (xp, 3 per group).
template <typename T>
__global__ void halo_peak_pos_kernel(const T *__restrict__ pos, int64_t G, Scale sc,
                                     const unsigned long long *__restrict__ pkey,
                                     const unsigned long long *__restrict__ cnt, long long *__restrict__ xp)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = cnt[g] ? (int64_t)(0xFFFFFFFFu - (uint32_t)pkey[g]) : 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) xp[3 * g + d] = cnt[g] ? fixed_of(pos[3 * p + d], sc.hi, sc.lo, sc.s) : 0;
    }
}

template <typename T>
__global__ void halo_sum_kernel(const T *__restrict__ pos, const int32_t *__restrict__ group, int64_t n, int64_t G,
                                Scale sc, const long long *__restrict__ xp, unsigned long long *__restrict__ sum)
{
    const int lane = threadIdx.x & 31;
    const WarpSpan ws;
    for (int64_t w0 = ws.w * kHaloSpan; w0 < n; w0 += ws.nw * kHaloSpan) {
        int32_t cg = -1;
        long long cs[3] = {0, 0, 0};
        for (int t = 0; t < kHaloSteps; t += kHaloU) {
            int32_t g[kHaloU];
#pragma unroll
            for (int u = 0; u < kHaloU; ++u) {
                const int64_t i = w0 + (int64_t)(t + u) * 32 + lane;
                g[u] = i < n ? group[i] : -1;
                if (g[u] >= G) g[u] = -1;
            }
            T x[kHaloU][3];
            long long c[kHaloU][3];
#pragma unroll
            for (int u = 0; u < kHaloU; ++u) {
                const int64_t i = w0 + (int64_t)(t + u) * 32 + lane;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    x[u][d] = g[u] >= 0 ? pos[3 * i + d] : T(0);
                    c[u][d] = g[u] >= 0 ? xp[3 * (int64_t)g[u] + d] : 0;
                }
            }
#pragma unroll
            for (int u = 0; u < kHaloU; ++u) {
                const int32_t gg = g[u];
                if (!__any_sync(0xffffffffu, gg >= 0)) continue;
                const uint32_t heads = run_heads((int64_t)gg, lane);
                long long o[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    o[d] = gg >= 0 ? wrap_units(fixed_of(x[u][d], sc.hi, sc.lo, sc.s) - c[u][d]) : 0;
                    o[d] = run_sum_i42(heads, lane, o[d]);   // |o| <= 2^31
                }
                if (lane == 0 && cg >= 0) {
                    if (gg == cg) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) o[d] += cs[d];
                    } else {
#pragma unroll
                        for (int d = 0; d < 3; ++d) atomicAdd(&sum[3 * (int64_t)cg + d], (unsigned long long)cs[d]);
                    }
                }
                const int last = last_head(heads);
                if (gg >= 0 && ((heads >> lane) & 1u) && lane != last)
#pragma unroll
                    for (int d = 0; d < 3; ++d) atomicAdd(&sum[3 * (int64_t)gg + d], (unsigned long long)o[d]);
                cg = __shfl_sync(0xffffffffu, gg, last);
#pragma unroll
                for (int d = 0; d < 3; ++d) cs[d] = __shfl_sync(0xffffffffu, o[d], last);
            }
        }
        if (lane == 0 && cg >= 0)
#pragma unroll
            for (int d = 0; d < 3; ++d) atomicAdd(&sum[3 * (int64_t)cg + d], (unsigned long long)cs[d]);
    }
}

// Per group: count, peak, the centre in units (cen, in [0, 2^32); it holds
// the peak's coordinates on entry) and in box coordinates (com).
__global__ void halo_centre_kernel(int64_t G, double box, const unsigned long long *__restrict__ pkey,
                                   const unsigned long long *__restrict__ cnt,
                                   const unsigned long long *__restrict__ sum, long long *__restrict__ cen,
                                   int64_t *__restrict__ count, uint32_t *__restrict__ peak, double *__restrict__ com)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = cnt[g];
        count[g] = (int64_t)c;
        peak[g] = c ? 0xFFFFFFFFu - (uint32_t)pkey[g] : 0u;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double u = 0.0;
            if (c) {
                u = (double)cen[3 * g + d] + (double)(long long)sum[3 * g + d] / (double)c;
                if (u < 0.0) u += (double)kUnits;
                if (u >= (double)kUnits) u -= (double)kUnits;
            }
            cen[3 * g + d] = __double2ll_rn(u) & (kUnits - 1);
            double x = u * (box / (double)kUnits);
            if (x >= box) x -= box;
            com[3 * g + d] = x;
        }
    }
}

// Largest squared member distance from the centre, in units^2: every
// wrapped component is at most 2^31, so the sum of three squares fits
// uint64.
template <typename T>
__global__ void halo_radius_kernel(const T *__restrict__ pos, const int32_t *__restrict__ group, int64_t n, int64_t G,
                                   Scale sc, const long long *__restrict__ cen, unsigned long long *__restrict__ r2max)
{
    const int lane = threadIdx.x & 31;
    const WarpSpan ws;
    for (int64_t w0 = ws.w * kHaloSpan; w0 < n; w0 += ws.nw * kHaloSpan) {
        int32_t cg = -1;
        unsigned long long cb = 0;
        for (int t = 0; t < kHaloSteps; t += kHaloU) {
            int32_t g[kHaloU];
#pragma unroll
            for (int u = 0; u < kHaloU; ++u) {
                const int64_t i = w0 + (int64_t)(t + u) * 32 + lane;
                g[u] = i < n ? group[i] : -1;
                if (g[u] >= G) g[u] = -1;
            }
            T x[kHaloU][3];
            long long c[kHaloU][3];
#pragma unroll
            for (int u = 0; u < kHaloU; ++u) {
                const int64_t i = w0 + (int64_t)(t + u) * 32 + lane;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    x[u][d] = g[u] >= 0 ? pos[3 * i + d] : T(0);
                    c[u][d] = g[u] >= 0 ? cen[3 * (int64_t)g[u] + d] : 0;
                }
            }
#pragma unroll
            for (int u = 0; u < kHaloU; ++u) {
                const int32_t gg = g[u];
                if (!__any_sync(0xffffffffu, gg >= 0)) continue;
                const uint32_t heads = run_heads((int64_t)gg, lane);
                unsigned long long b = 0;
                if (gg >= 0) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const long long dx = wrap_units(fixed_of(x[u][d], sc.hi, sc.lo, sc.s) - c[u][d]);
                        b += (unsigned long long)(dx * dx);
                    }
                }
                b = run_max(heads, lane, b);
                if (lane == 0 && cg >= 0) {
                    if (gg == cg) b = b > cb ? b : cb;
                    else atomicMax(&r2max[cg], cb);
                }
                const int last = last_head(heads);
                if (gg >= 0 && ((heads >> lane) & 1u) && lane != last) atomicMax(&r2max[gg], b);
                cg = __shfl_sync(0xffffffffu, gg, last);
                cb = __shfl_sync(0xffffffffu, b, last);
            }
        }
        if (lane == 0 && cg >= 0) atomicMax(&r2max[cg], cb);
    }
}

__global__ void halo_rmax_kernel(int64_t G, double box, const unsigned long long *__restrict__ r2max,
                                 double *__restrict__ rmax)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x)
        rmax[g] = sqrt((double)r2max[g]) * (box / (double)kUnits);
}

template <typename T>
int halo_stats_t(hop_ctx *c, const T *pos, const float *dens, const int32_t *group, int64_t n, int64_t G,
                 double box, int64_t *count, uint32_t *peak, double *com, double *rmax)
{
    // scratch: peak keys, counts, squared radii, offset sums (3), centres in units (3)
    char *s = (char *)ctx_buf(c, S_HALO, (size_t)G * 9 * 8);
    if (!s) return HOP_ENOMEM;
    unsigned long long *pkey = (unsigned long long *)s, *cnt = pkey + G, *r2 = cnt + G, *sum = r2 + G;
    long long *cen = (long long *)(sum + 3 * G);
    HOP_CUDA(c, cudaMemsetAsync(s, 0, (size_t)G * 6 * 8, c->stream));
    Scale sc;
    sc.s = (double)kUnits / box;
    sc.hi = (float)sc.s;
    sc.lo = (float)(sc.s - (double)sc.hi);
    halo_peak_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(dens, group, n, G, pkey, cnt, c->d_err);
    HOP_LAUNCH(c);
    halo_peak_pos_kernel<T><<<grid_for(c, G), 256, 0, c->stream>>>(pos, G, sc, pkey, cnt, cen);
    HOP_LAUNCH(c);
    halo_sum_kernel<T><<<grid_for(c, n), 256, 0, c->stream>>>(pos, group, n, G, sc, cen, sum);
    HOP_LAUNCH(c);
    halo_centre_kernel<<<grid_for(c, G), 256, 0, c->stream>>>(G, box, pkey, cnt, sum, cen, count, peak, com);
    HOP_LAUNCH(c);
    halo_radius_kernel<T><<<grid_for(c, n), 256, 0, c->stream>>>(pos, group, n, G, sc, cen, r2);
    HOP_LAUNCH(c);
    halo_rmax_kernel<<<grid_for(c, G), 256, 0, c->stream>>>(G, box, r2, rmax);
    HOP_LAUNCH(c);
    return HOP_OK;
}

}  // namespace

extern "C" int hop_halo_stats(hop_ctx *c, const void *pos, int32_t pos_is_f64, const float *dens,
                              const int32_t *group, int64_t n, int64_t n_groups, double box, int64_t *count,
                              uint32_t *peak, double *com, double *rmax)
{
    if (!c) return HOP_EINVAL;
    c->err.clear();
    if (!pos || !dens || !group || n <= 0 || n_groups < 0)
        return ctx_fail(c, HOP_EINVAL, "pos, dens, group and n > 0 are required");
    if (!(box > 0)) return ctx_fail(c, HOP_EINVAL, "box must be positive");
    if (n_groups == 0) return HOP_OK;
    if (!count || !peak || !com || !rmax) return ctx_fail(c, HOP_EINVAL, "outputs are required");
    HOP_CUDA(c, cudaSetDevice(c->device));
    HOP_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    const int rc = pos_is_f64
                       ? halo_stats_t<double>(c, (const double *)pos, dens, group, n, n_groups, box, count, peak,
                                              com, rmax)
                       : halo_stats_t<float>(c, (const float *)pos, dens, group, n, n_groups, box, count, peak,
                                             com, rmax);
    if (rc) return rc;
    HOP_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    const int e = ctx_check_device_error(c);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]) != cudaSuccess) cudaGetLastError();
    c->stats.ms_total = ms;
    return e;
}
