// Stable LSD radix sort of (key, int32 value) pairs with 8-bit digits.
// Per pass: per-tile digit histograms (digit-major), one device-wide exclusive
// scan of them, and a stable scatter where each warp ranks its keys with
// match.any and the warps of a tile are ordered by a per-digit prefix.
// The element count may live on the device (grids are sized by capacity and
// tiles past the count do nothing), so the sort needs no host round trip.
#include "internal.h"

namespace rl {

namespace {
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                 // keys per lane
constexpr int kTile = kThreads * kItems;  // keys per block
constexpr int kRadix = 256;

__device__ __forceinline__ int64_t bounded_count(int64_t max_n, const int32_t *d_count)
{
    if (!d_count) return max_n;
    int64_t c = *d_count;
    if (c < 0) c = 0;
    return c < max_n ? c : max_n;
}

template <typename K>
__global__ void __launch_bounds__(kThreads)
    hist_kernel(const K *__restrict__ keys, int64_t max_n, const int32_t *d_count, int shift,
                int32_t *__restrict__ hist, int nblocks)
{
    __shared__ int32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t n = bounded_count(max_n, d_count);
    const int64_t base = (int64_t)blockIdx.x * kTile;
    if (base < n) {
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
            if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 0xFFu], 1);
        }
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(kThreads)
    scatter_kernel(const K *__restrict__ keys_in, const int32_t *__restrict__ vals_in,
                   K *__restrict__ keys_out, int32_t *__restrict__ vals_out, int64_t max_n,
                   const int32_t *d_count, int shift, const int32_t *__restrict__ offsets,
                   int nblocks)
{
    __shared__ int32_t wcnt[kWarps][kRadix];
    const int64_t n = bounded_count(max_n, d_count);
    const int64_t block_base = (int64_t)blockIdx.x * kTile;
    if (block_base >= n) return;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = block_base + (int64_t)warp * (32 * kItems);
    const uint32_t lt = lanemask_lt();
    K k[kItems];
    int32_t v[kItems];
    int dig[kItems], rank[kItems];
#pragma unroll
    for (int s = 0; s < kItems; ++s) {
        int64_t i = base + s * 32 + lane;
        bool ok = i < n;
        k[s] = ok ? keys_in[i] : K(0);
        v[s] = ok ? vals_in[i] : 0;
        dig[s] = ok ? (int)((uint32_t)(k[s] >> shift) & 0xFFu) : kRadix;
    }
#pragma unroll
    for (int s = 0; s < kItems; ++s) {
        uint32_t peers = __match_any_sync(0xffffffffu, dig[s]);
        int leader = __ffs(peers) - 1;
        int before = dig[s] < kRadix ? wcnt[warp][dig[s]] : 0;
        __syncwarp();
        if (lane == leader && dig[s] < kRadix) wcnt[warp][dig[s]] = before + __popc(peers);
        __syncwarp();
        rank[s] = before + __popc(peers & lt);
    }
    __syncthreads();
    {   // per-digit exclusive prefix over the warps of this tile
        const int d = threadIdx.x;
        int32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            int32_t c = wcnt[w][d];
            wcnt[w][d] = acc + offsets[(int64_t)d * nblocks + blockIdx.x];
            acc += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kItems; ++s) {
        if (dig[s] < kRadix) {
            int32_t pos = wcnt[warp][dig[s]] + rank[s];
            keys_out[pos] = k[s];
            vals_out[pos] = v[s];
        }
    }
}

template <typename K>
cudaError_t radix_sort(K *keys, K *keys_alt, int32_t *vals, int32_t *vals_alt, int64_t max_n,
                       const int32_t *d_count, int end_bit, SortScratch &s, cudaStream_t st,
                       int *which)
{
    *which = 0;
    if (max_n <= 0 || end_bit <= 0) return cudaSuccess;
    int64_t nb64 = sort_blocks_needed(max_n);
    if (nb64 > s.max_blocks || nb64 > 0x7fffffff) return cudaErrorInvalidValue;
    int nb = (int)nb64;
    K *kin = keys, *kout = keys_alt;
    int32_t *vin = vals, *vout = vals_alt;
    for (int shift = 0; shift < end_bit; shift += 8) {
        hist_kernel<K><<<nb, kThreads, 0, st>>>(kin, max_n, d_count, shift, s.hist, nb);
        note_launch();
        cudaError_t e = scan_exclusive(s.hist, s.hist, (int64_t)kRadix * nb, nullptr, nullptr,
                                       s.scan, st);
        if (e != cudaSuccess) return e;
        scatter_kernel<K><<<nb, kThreads, 0, st>>>(kin, vin, kout, vout, max_n, d_count, shift,
                                                    s.hist, nb);
        note_launch();
        K *tk = kin;
        kin = kout;
        kout = tk;
        int32_t *tv = vin;
        vin = vout;
        vout = tv;
        *which ^= 1;
    }
    return cudaGetLastError();
}
} // namespace

int64_t sort_blocks_needed(int64_t max_n) { return (max_n + kTile - 1) / kTile; }

cudaError_t radix_sort_u32(uint32_t *keys, uint32_t *keys_alt, int32_t *vals, int32_t *vals_alt,
                           int64_t max_n, const int32_t *d_count, int end_bit, SortScratch &s,
                           cudaStream_t st, int *which)
{
    return radix_sort<uint32_t>(keys, keys_alt, vals, vals_alt, max_n, d_count, end_bit, s, st,
                                which);
}

cudaError_t radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, int32_t *vals, int32_t *vals_alt,
                           int64_t max_n, const int32_t *d_count, int end_bit, SortScratch &s,
                           cudaStream_t st, int *which)
{
    return radix_sort<uint64_t>(keys, keys_alt, vals, vals_alt, max_n, d_count, end_bit, s, st,
                                which);
}

} // namespace rl
