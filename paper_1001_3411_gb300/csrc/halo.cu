// Halo statistics: once the halos are known, Parallel HOP computes for
// each its dark matter mass, centre of mass and maximum radius (Sec. 3,
// end of the merging description).  Particle masses are equal, so the mass
// is the member count.  In the periodic box the centre of mass is taken
// about the halo's peak particle (its densest member, then the smaller
// index): members' minimum-image offsets from the peak are averaged and
// added to the peak's position, wrapped into [0, box).  The offsets are
// summed in fixed point (2^-32 of the box, int64 atomics), so the centres do
// not depend on the order of the sums and lie within 2^-33 of the box of
// the exact mean.  The maximum
// radius is the largest minimum-image distance from that centre to a member.
//
// Four grid-stride passes over the particles, each HBM-bound: peak keys and
// counts, offset sums, (per group) the centre, then the radii.  A warp
// reduces each run of consecutive lanes holding the same group with a
// segmented shuffle scan (five steps), so one atomic per run reaches
// memory; members of a halo are mostly consecutive in the input.
#include "hop_internal.cuh"

#include <algorithm>

namespace {

__device__ __forceinline__ double min_image_d(double dx, double box)
{
    if (dx > 0.5 * box) return dx - box;
    if (dx < -0.5 * box) return dx + box;
    return dx;
}

template <typename T> __device__ __forceinline__ double coord(const T *pos, int64_t i, int d)
{
    return (double)pos[3 * i + d];
}

__global__ void halo_peak_kernel(const float *__restrict__ dens, const int32_t *__restrict__ group, int64_t n,
                                 int64_t G, unsigned long long *__restrict__ pkey,
                                 unsigned long long *__restrict__ count, uint32_t *__restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        int32_t g = i < n ? group[i] : -1;
        if (g >= G) {
            atomicOr(err, kErrBadIndex);
            g = -1;
        }
        if (!__any_sync(0xffffffffu, g >= 0)) continue;
        const uint32_t heads = run_heads((int64_t)g, lane);
        const unsigned long long key =
            g >= 0 ? ((unsigned long long)__float_as_uint(dens[i]) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)i)
                   : 0ull;
        const unsigned long long best = run_max(heads, lane, key);
        if (g >= 0 && ((heads >> lane) & 1u)) {
            atomicMax(&pkey[g], best);
            atomicAdd(&count[g], (unsigned long long)run_len(heads, lane));
        }
    }
}

template <typename T>
__global__ void halo_sum_kernel(const T *__restrict__ pos, const int32_t *__restrict__ group, int64_t n, int64_t G,
                                double box, const unsigned long long *__restrict__ pkey,
                                unsigned long long *__restrict__ sum)
{
    const int lane = threadIdx.x & 31;
    const double scale = 4294967296.0 / box;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        int32_t g = i < n ? group[i] : -1;
        if (g >= G) g = -1;
        if (!__any_sync(0xffffffffu, g >= 0)) continue;
        const uint32_t heads = run_heads((int64_t)g, lane);
        long long o[3] = {0, 0, 0};
        if (g >= 0) {
            const int64_t p = (int64_t)(0xFFFFFFFFu - (uint32_t)pkey[g]);
#pragma unroll
            for (int d = 0; d < 3; ++d)
                o[d] = __double2ll_rn(min_image_d(coord(pos, i, d) - coord(pos, p, d), box) * scale);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) o[d] = run_sum<long long>(heads, lane, o[d]);
        if (g >= 0 && ((heads >> lane) & 1u))
            for (int d = 0; d < 3; ++d) atomicAdd(&sum[3 * (int64_t)g + d], (unsigned long long)o[d]);
    }
}

template <typename T>
__global__ void halo_centre_kernel(const T *__restrict__ pos, int64_t G, double box,
                                   const unsigned long long *__restrict__ pkey,
                                   const unsigned long long *__restrict__ cnt,
                                   const unsigned long long *__restrict__ sum,
                                   int64_t *__restrict__ count, uint32_t *__restrict__ peak, double *__restrict__ com)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = cnt[g];
        count[g] = (int64_t)c;
        const uint32_t p = c ? 0xFFFFFFFFu - (uint32_t)pkey[g] : 0u;
        peak[g] = p;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double mean = (double)(long long)sum[3 * g + d] / (double)c * (box / 4294967296.0);
            double x = c ? coord(pos, (int64_t)p, d) + mean : 0.0;
            if (x < 0.0) x += box;
            if (x >= box) x -= box;
            com[3 * g + d] = x;
        }
    }
}

template <typename T>
__global__ void halo_radius_kernel(const T *__restrict__ pos, const int32_t *__restrict__ group, int64_t n, int64_t G,
                                   double box, const double *__restrict__ com, unsigned long long *__restrict__ rbits)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        int32_t g = i < n ? group[i] : -1;
        if (g >= G) g = -1;
        if (!__any_sync(0xffffffffu, g >= 0)) continue;
        const uint32_t heads = run_heads((int64_t)g, lane);
        unsigned long long b = 0;
        if (g >= 0) {
            double r2 = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double dx = min_image_d(coord(pos, i, d) - com[3 * (int64_t)g + d], box);
                r2 += dx * dx;
            }
            // non-negative doubles order like their bit patterns
            b = (unsigned long long)__double_as_longlong(sqrt(r2));
        }
        b = run_max(heads, lane, b);
        if (g >= 0 && ((heads >> lane) & 1u)) atomicMax(&rbits[g], b);
    }
}

__global__ void halo_rmax_kernel(int64_t G, const unsigned long long *__restrict__ rbits, double *__restrict__ rmax)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x)
        rmax[g] = __longlong_as_double((long long)rbits[g]);
}

template <typename T>
int halo_stats_t(hop_ctx *c, const T *pos, const float *dens, const int32_t *group, int64_t n, int64_t G,
                 double box, int64_t *count, uint32_t *peak, double *com, double *rmax)
{
    // scratch: peak keys, counts, offset sums (3), radius bits
    char *s = (char *)ctx_buf(c, S_HALO, (size_t)G * 6 * 8);
    if (!s) return HOP_ENOMEM;
    unsigned long long *pkey = (unsigned long long *)s, *cnt = pkey + G, *rbits = cnt + G, *sum = rbits + G;
    HOP_CUDA(c, cudaMemsetAsync(s, 0, (size_t)G * 6 * 8, c->stream));
    halo_peak_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(dens, group, n, G, pkey, cnt, c->d_err);
    HOP_LAUNCH(c);
    halo_sum_kernel<T><<<grid_for(c, n), 256, 0, c->stream>>>(pos, group, n, G, box, pkey, sum);
    HOP_LAUNCH(c);
    halo_centre_kernel<T><<<grid_for(c, G), 256, 0, c->stream>>>(pos, G, box, pkey, cnt, sum, count, peak, com);
    HOP_LAUNCH(c);
    halo_radius_kernel<T><<<grid_for(c, n), 256, 0, c->stream>>>(pos, group, n, G, box, com, rbits);
    HOP_LAUNCH(c);
    halo_rmax_kernel<<<grid_for(c, G), 256, 0, c->stream>>>(G, rbits, rmax);
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
