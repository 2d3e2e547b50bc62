// Device-wide exclusive scan of int32 with int64 carries, in one pass (decoupled
// look-back): a grid of at most the resident blocks, each taking the next tile by
// ticket until none is left (capacity-sized scans of short inputs then launch no
// waves of idle blocks), stages it in shared memory
// (coalesced global reads and writes), sums it, publishes the tile sum, then its
// first warp reads the states of the 32 preceding tiles at once and adds their
// published sums back to the nearest one that has published its inclusive prefix
// (further windows of 32 if none has), and the block publishes its own inclusive
// prefix. A block only waits for tiles with smaller tickets, which are held by
// blocks already running that publish their sums before they wait themselves, so
// every wait ends; each is still bounded (kSpin rounds, then RELEARN_ERR_TIMEOUT in
// the status word and no block waits any more).
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

constexpr int32_t kAgg = 1, kInc = 2;
constexpr int kSpin = 1 << 16;

// flags[0]: ticket counter, flags[1]: abort flag, flags[2]: blocks finished, flags[3 + t]:
// state of tile t; all zero at launch. The last block to finish (every other block has
// made its last access by then) sets them back to zero, so scans need no memset.
// agg[t], inc[t]: tile t's sum and inclusive prefix.
__device__ __forceinline__ void scan_tile(const int32_t *in, int32_t *out, int64_t n, int64_t t,
                                          int64_t last_tile, int32_t *flags, int64_t *agg,
                                          int64_t *inc, int64_t *d_total, int32_t *status,
                                          int32_t *tile, int64_t &s_prefix)
{
    const int64_t base = t * kTile;
    for (int k = 0; k < kItems; ++k) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
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
    const int64_t incl = block_inclusive<kThreads>(s, &tot);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const volatile int32_t *state = flags + 3;
        int64_t prefix = 0;
        if (t > 0) {
            if (lane == 0) {
                agg[t] = tot;
                __threadfence();
                atomicExch(&flags[3 + t], kAgg);
            }
            // the 256 nearest predecessors in one round: lane l reads j = t-1-l-32k,
            // k < kWin; wait until all have published, then add the aggregates back to
            // the nearest inclusive prefix among them (further tiles window by window)
            constexpr int kWin = 8;
            int32_t f[kWin];
            bool ready = false;
            for (int spin = 0; spin < kSpin; ++spin) {
                bool mine = true;
#pragma unroll
                for (int k = 0; k < kWin; ++k) {
                    const int64_t j = t - 1 - lane - 32 * k;
                    f[k] = j < 0 ? kInc : state[j];
                    mine = mine && f[k] != 0;
                }
                ready = __all_sync(0xffffffffu, mine);
                if (ready || *(volatile int32_t *)&flags[1]) break;
            }
            if (!ready) {
                if (lane == 0) {
                    if (status) set_status(status, RELEARN_ERR_TIMEOUT);
                    atomicExch(&flags[1], 1);
                }
            } else {
                __threadfence();
                // nearest predecessor (largest index) holding an inclusive prefix
                int64_t jinc = -1;
#pragma unroll
                for (int k = 0; k < kWin; ++k) {
                    const int64_t j = t - 1 - lane - 32 * k;
                    if (j >= 0 && f[k] == kInc && j > jinc) jinc = j;
                }
                for (int o = 16; o; o >>= 1) {
                    const int64_t other = __shfl_xor_sync(0xffffffffu, jinc, o);
                    jinc = other > jinc ? other : jinc;
                }
                int64_t w = 0;
#pragma unroll
                for (int k = 0; k < kWin; ++k) {
                    const int64_t j = t - 1 - lane - 32 * k;
                    if (j < 0 || j < jinc) continue;
                    w += j == jinc ? *(const volatile int64_t *)&inc[j]
                                   : *(const volatile int64_t *)&agg[j];
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                prefix = w;
                // no inclusive prefix within reach: walk on, one window of 32 at a time
                const bool more = jinc < 0 && t - 1 - 32 * kWin >= 0;
                for (int64_t j0 = t - 1 - 32 * kWin; more; j0 -= 32) {
                    const int64_t j = j0 - lane; // this lane's predecessor (j < 0: zero)
                    int32_t g = j < 0 ? kInc : 0;
                    bool rd = false;
                    for (int spin = 0; spin < kSpin; ++spin) {
                        if (j >= 0) g = state[j];
                        rd = __all_sync(0xffffffffu, g != 0);
                        if (rd || *(volatile int32_t *)&flags[1]) break;
                    }
                    if (!rd) { // gave up (or another block did): report, stop waiting
                        if (lane == 0) {
                            if (status) set_status(status, RELEARN_ERR_TIMEOUT);
                            atomicExch(&flags[1], 1);
                        }
                        break;
                    }
                    __threadfence();
                    const uint32_t incm = __ballot_sync(0xffffffffu, g == kInc);
                    const int stop = incm ? __ffs(incm) - 1 : 32; // nearest inclusive prefix
                    int64_t v = 0;
                    if (j >= 0 && lane < stop) v = *(const volatile int64_t *)&agg[j];
                    if (j >= 0 && lane == stop) v = *(const volatile int64_t *)&inc[j];
#pragma unroll
                    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    prefix += v;
                    if (incm) break;
                }
            }
        }
        if (lane == 0) {
            inc[t] = prefix + tot;
            __threadfence();
            atomicExch(&flags[3 + t], kInc);
            s_prefix = prefix;
            if (t == last_tile && d_total) *d_total = prefix + tot;
        }
    }
    __syncthreads();
    int64_t run = s_prefix + incl - s;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        tile[threadIdx.x * kItems + k] = (int32_t)run;
        run += v[k];
    }
    __syncthreads();
    for (int k = 0; k < kItems; ++k) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) out[i] = tile[k * kThreads + threadIdx.x];
    }
}

__global__ void __launch_bounds__(kThreads)
    scan_kernel(const int32_t *in, int32_t *out, int64_t max_n, const int32_t *d_count,
                int32_t *flags, int64_t *agg, int64_t *inc, int64_t *d_total, int32_t *status)
{
    __shared__ int32_t tile[kTile];
    __shared__ int64_t s_prefix;
    __shared__ int32_t s_t, s_last;
    const int64_t max_tiles = max_n > 0 ? (max_n + kTile - 1) / kTile : 1;
    if (threadIdx.x == 0) s_t = atomicAdd(&flags[0], 1);
    __syncthreads();
    const int64_t n = bounded_count(max_n, d_count);
    // tiles past the last element (capacities are sized for the largest input) have
    // nothing to do, and no tile that has elements looks back at them
    const int64_t last_tile = n > 0 ? (n - 1) / kTile : 0;
    // a persistent grid: each block takes tiles by ticket until they run out (a tile
    // only waits for smaller tickets, held by blocks already running)
    for (int64_t t = s_t; t <= last_tile;) {
        scan_tile(in, out, n, t, last_tile, flags, agg, inc, d_total, status, tile, s_prefix);
        __syncthreads();
        if (threadIdx.x == 0) s_t = atomicAdd(&flags[0], 1);
        __syncthreads();
        t = s_t;
    }
    // the last block to finish clears the ticket, abort flag, counter and tile states
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&flags[2], 1) == (int32_t)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int64_t j = threadIdx.x; j < max_tiles; j += blockDim.x) flags[3 + j] = 0;
        if (threadIdx.x == 0) {
            flags[0] = 0;
            flags[1] = 0;
            flags[2] = 0;
        }
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

int64_t scan_grid_cap(int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_kernel, kThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return (int64_t)per_sm * (num_sms > 0 ? num_sms : 1);
}

cudaError_t scan_exclusive(const int32_t *in, int32_t *out, int64_t max_n, const int32_t *d_count,
                           int64_t *d_total, ScanScratch &s, cudaStream_t st)
{
    int64_t nb = scan_blocks_needed(max_n);
    if (nb == 0) nb = 1;
    if (nb > s.max_blocks) return cudaErrorInvalidValue;
    // a grid of resident blocks at most: they take the tiles by ticket
    const int64_t grid = nb < s.grid_cap ? nb : s.grid_cap;
    // s.flags is zero here: zeroed at allocation and cleared by every scan's last block
    scan_kernel<<<(unsigned)grid, kThreads, 0, st>>>(in, out, max_n, d_count, s.flags,
                                                     s.block_sums, s.block_sums + nb, d_total,
                                                     s.status);
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
