// Single-pass exclusive scan of a pair of int32 sequences over the same index range
// (two independent prefix sums, int64 carries), with the consumer fused in: each
// element's exclusive prefixes go straight to a caller-supplied epilogue instead of
// to an array that a further kernel would read back.
//
// Decoupled look-back as in scan.cu: each block takes the next tile by ticket,
// stages it in shared memory (coalesced reads), sums it, publishes the tile sums,
// then its first warp reads the states of the 256 preceding tiles at once and adds
// their published sums back to the nearest one that has published its inclusive
// prefixes (further windows of 32 if none has). A block only waits for tiles with
// smaller tickets, which are held by blocks already running that publish their sums
// before they wait themselves, so every wait ends; each is still bounded (kPairSpin
// rounds, then RELEARN_ERR_TIMEOUT in the status word and no block waits any more).
//
// Op supplies:
//   void prologue(int64_t i, int64_t stride) once for every thread, i = its index in the
//                                            grid, stride = the grid's thread count
//                                            (side work that finish() may rely on)
//   int2 load(int64_t k)                     the pair of element k (k < n)
//   void emit(int64_t k, int64_t a, int64_t b, int2 v)
//                                            element k's exclusive prefixes and its
//                                            pair (k < n), one call per element
//   void store_totals(int64_t a, int64_t b)  the two totals, once (the last tile)
//   void finish()                            once, by one thread of the last block to
//                                            finish (every other block is done, and
//                                            the totals are stored)
// flags: [tiles + 3] zero at launch and left zero (the last block clears them);
// sums: [4 * tiles] int64 scratch; stall_tile: a tile that publishes nothing (a test
// of the bounded waits; -1: none).
#pragma once

#include "internal.h"

namespace rl {

namespace pair_scan {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
constexpr int kPad = kTile + kTile / 32; // element e at e + e / 32 (bank spread)
constexpr int32_t kAgg = 1, kInc = 2;
constexpr int kPairSpin = 1 << 16;
constexpr int kWin = 8; // the first look-back round covers 32 * kWin tiles

__device__ __forceinline__ longlong2 ll2_add(longlong2 a, longlong2 b)
{
    return make_longlong2(a.x + b.x, a.y + b.y);
}

__device__ __forceinline__ longlong2 ll2_shfl_up(longlong2 v, int o)
{
    return make_longlong2(__shfl_up_sync(0xffffffffu, v.x, o),
                          __shfl_up_sync(0xffffffffu, v.y, o));
}

__device__ __forceinline__ longlong2 ll2_xor_sum(longlong2 v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1)
        v = make_longlong2(v.x + __shfl_xor_sync(0xffffffffu, v.x, o),
                           v.y + __shfl_xor_sync(0xffffffffu, v.y, o));
    return v;
}

__device__ __forceinline__ longlong2 ll2_load_volatile(const longlong2 *p)
{
    const volatile long long *q = reinterpret_cast<const volatile long long *>(p);
    return make_longlong2(q[0], q[1]);
}

// Inclusive block scan of pairs (256 threads); *total = block sums.
__device__ __forceinline__ longlong2 ll2_block_inclusive(longlong2 v, longlong2 *total,
                                                         longlong2 *wt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const longlong2 t = ll2_shfl_up(v, o);
        if (lane >= o) v = ll2_add(v, t);
    }
    if (lane == 31) wt[warp] = v;
    __syncthreads();
    if (warp == 0) {
        longlong2 w = lane < 8 ? wt[lane] : make_longlong2(0, 0);
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const longlong2 t = ll2_shfl_up(w, o);
            if (lane >= o) w = ll2_add(w, t);
        }
        if (lane < 8) wt[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v = ll2_add(v, wt[warp - 1]);
    *total = wt[7];
    __syncthreads();
    return v;
}

// Prefix of tile t from its predecessors (first warp; every lane returns it).
__device__ __forceinline__ longlong2 look_back(int64_t t, const volatile int32_t *state,
                                               int32_t *flags, const longlong2 *agg,
                                               const longlong2 *inc, int32_t *status)
{
    const int lane = threadIdx.x & 31;
    int32_t f[kWin];
    bool ready = false;
    for (int spin = 0; spin < kPairSpin; ++spin) {
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
    if (!ready) { // gave up (or another block did): report, stop waiting
        if (lane == 0) {
            if (status) set_status(status, RELEARN_ERR_TIMEOUT);
            atomicExch(&flags[1], 1);
        }
        return make_longlong2(0, 0);
    }
    __threadfence();
    // nearest predecessor (largest index) holding inclusive prefixes
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
    longlong2 w = make_longlong2(0, 0);
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
        const int64_t j = t - 1 - lane - 32 * k;
        if (j < 0 || j < jinc) continue;
        w = ll2_add(w, ll2_load_volatile(j == jinc ? &inc[j] : &agg[j]));
    }
    longlong2 prefix = ll2_xor_sum(w);
    // no inclusive prefix within reach: walk on, one window of 32 at a time
    const bool more = jinc < 0 && t - 1 - 32 * kWin >= 0;
    for (int64_t j0 = t - 1 - 32 * kWin; more; j0 -= 32) {
        const int64_t j = j0 - lane; // this lane's predecessor (j < 0: zero)
        int32_t g = j < 0 ? kInc : 0;
        bool rd = false;
        for (int spin = 0; spin < kPairSpin; ++spin) {
            if (j >= 0) g = state[j];
            rd = __all_sync(0xffffffffu, g != 0);
            if (rd || *(volatile int32_t *)&flags[1]) break;
        }
        if (!rd) {
            if (lane == 0) {
                if (status) set_status(status, RELEARN_ERR_TIMEOUT);
                atomicExch(&flags[1], 1);
            }
            break;
        }
        __threadfence();
        const uint32_t incm = __ballot_sync(0xffffffffu, g == kInc);
        const int stop = incm ? __ffs(incm) - 1 : 32; // nearest inclusive prefix
        longlong2 v = make_longlong2(0, 0);
        if (j >= 0 && lane < stop) v = ll2_load_volatile(&agg[j]);
        if (j >= 0 && lane == stop) v = ll2_load_volatile(&inc[j]);
        prefix = ll2_add(prefix, ll2_xor_sum(v));
        if (incm) break;
    }
    return prefix;
}

template <class Op>
__global__ void __launch_bounds__(kThreads)
    scan_pair_kernel(Op op, int64_t n, int32_t *flags, longlong2 *sums, int32_t *status,
                     int64_t stall_tile)
{
    __shared__ int32_t s_a[kPad], s_b[kPad]; // the tile's pairs, then their exclusive
                                             // prefixes within the tile
    __shared__ longlong2 s_wt[8];
    __shared__ longlong2 s_prefix;
    __shared__ int64_t s_tot[2];
    __shared__ int32_t s_t, s_last;
    if (threadIdx.x == 0) s_t = atomicAdd(&flags[0], 1);
    __syncthreads();
    const int64_t t = s_t;
    const int64_t tiles = (int64_t)gridDim.x;
    longlong2 *agg = sums, *inc = sums + tiles;
    const int64_t tile0 = t * kTile;
    op.prologue(t * kThreads + threadIdx.x, tiles * kThreads);
    // item-major loads (coalesced), thread-major scan
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int e = i * kThreads + threadIdx.x;
        const int64_t k = tile0 + e;
        const int2 v = k < n ? op.load(k) : make_int2(0, 0);
        s_a[e + e / 32] = v.x;
        s_b[e + e / 32] = v.y;
    }
    __syncthreads();
    int32_t va[kItems], vb[kItems];
    longlong2 s = make_longlong2(0, 0);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int e = threadIdx.x * kItems + i;
        va[i] = s_a[e + e / 32];
        vb[i] = s_b[e + e / 32];
        s.x += va[i];
        s.y += vb[i];
    }
    longlong2 tot;
    const longlong2 incl = ll2_block_inclusive(s, &tot, s_wt);
    const bool publish = t != stall_tile;
    if (threadIdx.x < 32) {
        longlong2 prefix = make_longlong2(0, 0);
        if (t > 0) {
            if (threadIdx.x == 0 && publish) {
                agg[t] = tot;
                __threadfence();
                atomicExch(&flags[3 + t], kAgg);
            }
            prefix = look_back(t, flags + 3, flags, agg, inc, status);
        }
        if (threadIdx.x == 0) {
            if (publish) {
                inc[t] = ll2_add(prefix, tot);
                __threadfence();
                atomicExch(&flags[3 + t], kInc);
            }
            s_prefix = prefix;
            if (t == tiles - 1) {
                s_tot[0] = prefix.x + tot.x;
                s_tot[1] = prefix.y + tot.y;
            }
        }
    }
    __syncthreads();
    // exclusive prefixes within the tile (a tile's sums fit in int32, as the outputs do)
    int64_t ra = incl.x - s.x, rb = incl.y - s.y;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int e = threadIdx.x * kItems + i;
        s_a[e + e / 32] = (int32_t)ra;
        s_b[e + e / 32] = (int32_t)rb;
        ra += va[i];
        rb += vb[i];
    }
    __syncthreads();
    const longlong2 base = s_prefix;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int e = i * kThreads + threadIdx.x;
        const int64_t k = tile0 + e;
        if (k < n) {
            // the element's pair: the next prefix (the tile sum after the last) minus its own
            const int32_t pa = s_a[e + e / 32], pb = s_b[e + e / 32];
            const int f = e + 1 + (e + 1) / 32;
            const int32_t na = e + 1 < kTile ? s_a[f] : (int32_t)tot.x;
            const int32_t nb = e + 1 < kTile ? s_b[f] : (int32_t)tot.y;
            op.emit(k, base.x + pa, base.y + pb, make_int2(na - pa, nb - pb));
        }
    }
    // the last block to finish: totals to the consumer, then clear the look-back state
    __syncthreads();
    if (threadIdx.x == 0) {
        if (t == tiles - 1) op.store_totals(s_tot[0], s_tot[1]);
        __threadfence();
        s_last = atomicAdd(&flags[2], 1) == (int32_t)tiles - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x == 0) op.finish();
        for (int64_t j = threadIdx.x; j < tiles; j += blockDim.x) flags[3 + j] = 0;
        if (threadIdx.x == 0) {
            flags[0] = 0;
            flags[1] = 0;
            flags[2] = 0;
        }
    }
}

} // namespace pair_scan

} // namespace rl
