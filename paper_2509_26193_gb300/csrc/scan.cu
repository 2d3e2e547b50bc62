// Device-wide exclusive scan of int32 with int64 block sums (reduce, spine,
// downsweep). Tiles are staged in shared memory so global traffic is coalesced.
#include "internal.h"

namespace rl {

namespace {
constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;

__device__ __forceinline__ int64_t bounded_count(int64_t max_n, const int32_t *d_count)
{
    if (!d_count) return max_n;
    int64_t c = *d_count;
    if (c < 0) c = 0;
    return c < max_n ? c : max_n;
}

__device__ __forceinline__ int64_t warp_inclusive(int64_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Inclusive scan over the block; *total receives the block sum.
template <int NT>
__device__ __forceinline__ int64_t block_inclusive(int64_t v, int64_t *total)
{
    __shared__ int64_t warp_tot[NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = warp_inclusive(v);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < NT / 32 ? warp_tot[lane] : 0;
        w = warp_inclusive(w);
        if (lane < NT / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    if (warp > 0) inc += warp_tot[warp - 1];
    *total = warp_tot[NT / 32 - 1];
    __syncthreads();
    return inc;
}

__global__ void __launch_bounds__(kThreads)
    scan_reduce_kernel(const int32_t *__restrict__ in, int64_t max_n, const int32_t *d_count,
                       int64_t *__restrict__ block_sums)
{
    const int64_t n = bounded_count(max_n, d_count);
    const int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t s = 0;
    if (base < n) {
#pragma unroll 4
        for (int k = 0; k < kItems; ++k) {
            int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
            if (i < n) s += in[i];
        }
    }
    int64_t tot;
    block_inclusive<kThreads>(s, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024)
    scan_spine_kernel(int64_t *__restrict__ block_sums, int64_t nb, int64_t *d_total)
{
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
        int64_t i = c0 + threadIdx.x;
        int64_t v = i < nb ? block_sums[i] : 0;
        int64_t tot;
        int64_t inc = block_inclusive<1024>(v, &tot);
        if (i < nb) block_sums[i] = carry + inc - v;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        block_sums[nb] = carry;
        if (d_total) *d_total = carry;
    }
}

__global__ void __launch_bounds__(kThreads)
    scan_down_kernel(const int32_t *in, int32_t *out, int64_t max_n, const int32_t *d_count,
                     const int64_t *__restrict__ block_sums)
{
    __shared__ int32_t tile[kTile];
    const int64_t n = bounded_count(max_n, d_count);
    const int64_t base = (int64_t)blockIdx.x * kTile;
    if (base >= n) return;
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        tile[k * kThreads + threadIdx.x] = i < n ? in[i] : 0;
    }
    __syncthreads();
    int32_t v[kItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = tile[threadIdx.x * kItems + k];
        s += v[k];
    }
    int64_t tot;
    int64_t run = block_inclusive<kThreads>(s, &tot) - s + block_sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        tile[threadIdx.x * kItems + k] = (int32_t)run;
        run += v[k];
    }
    __syncthreads();
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) out[i] = tile[k * kThreads + threadIdx.x];
    }
}

__global__ void fill_kernel(int32_t *p, int32_t v, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
} // namespace

int64_t scan_blocks_needed(int64_t max_n) { return (max_n + kTile - 1) / kTile; }

cudaError_t scan_exclusive(const int32_t *in, int32_t *out, int64_t max_n, const int32_t *d_count,
                           int64_t *d_total, ScanScratch &s, cudaStream_t st)
{
    int64_t nb = scan_blocks_needed(max_n);
    if (nb == 0) nb = 1;
    if (nb > s.max_blocks) return cudaErrorInvalidValue;
    scan_reduce_kernel<<<(unsigned)nb, kThreads, 0, st>>>(in, max_n, d_count, s.block_sums);
    note_launch();
    scan_spine_kernel<<<1, 1024, 0, st>>>(s.block_sums, nb, d_total);
    note_launch();
    scan_down_kernel<<<(unsigned)nb, kThreads, 0, st>>>(in, out, max_n, d_count, s.block_sums);
    note_launch();
    return cudaGetLastError();
}

cudaError_t fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, v, n);
    note_launch();
    return cudaGetLastError();
}

} // namespace rl
