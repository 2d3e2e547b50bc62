// Octree build and bottom-up update (Sec. III-B "Spatial octree" and
// "Division of work").
//
// Build: bounding box -> 30-bit Morton codes -> stable radix sort of (code, id)
// -> compressed octree in pre-order. A node is the root, a cell with >= 2
// non-empty child cells, or a depth-10 cell with >= 2 neurons (a bucket whose
// children are its neurons); every neuron is one leaf. A chain of single-child
// cells holds one neuron set and is stored once, at its deepest cell, which
// gives the same candidate (count, centroid) and the same restart point as the
// uncompressed octree. Nodes are laid out in pre-order with a skip link
// (`escape`) per node so that a search walks the tree without a stack.
//
// Reduce (bottom-up update): every node covers a contiguous Morton range, so its
// count and count-weighted position sums are differences of one exclusive prefix
// over the neurons in Morton order, formed in exact int64 fixed point (leaves and
// tile sums, then each tile's prefix); each inner node then takes its two prefix
// entries and rounds its centroid once to FP32 (see inner_sums).
#include <mutex>

#include "internal.h"

namespace rl {

namespace {

__device__ __forceinline__ uint32_t ordered(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Network of neuron (or Morton position) i: the b with off[b] <= i < off[b + 1].
__device__ __forceinline__ int32_t net_of(const int64_t *__restrict__ off, int32_t B, int64_t i)
{
    int32_t lo = 0, hi = B - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Network of Morton position s; one network keeps no per-position array.
__device__ __forceinline__ int32_t net_at(const int32_t *__restrict__ net, int64_t s)
{
    return net ? net[s] : 0;
}

// Per network b: d_ord[6b .. 6b+2] = min (ordered), d_ord[6b+3 .. 6b+5] = max; NaN
// coordinates are skipped. A warp whose 32 elements share a network reduces them
// before its atomics; elements at network boundaries go one by one.
__global__ void bbox_kernel(const float *__restrict__ x, const float *__restrict__ y,
                            const float *__restrict__ z, int64_t n,
                            const int64_t *__restrict__ off, int32_t B, uint32_t *d_ord)
{
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < n;
         w0 += wstride) {
        const int64_t i = w0 + lane;
        const bool ok = i < n;
        const int32_t b = ok ? (B == 1 ? 0 : net_of(off, B, i)) : -1;
        uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
        if (ok) {
            const float p[3] = {x[i], y[i], z[i]};
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (p[a] == p[a]) mn[a] = mx[a] = ordered(p[a]);
        }
        const int32_t b0 = __shfl_sync(0xffffffffu, b, 0);
        const int32_t b31 = __shfl_sync(0xffffffffu, ok ? b : b0, 31);
        if (b0 == b31) { // every valid lane is in network b0
#pragma unroll
            for (int a = 0; a < 3; ++a)
                for (int o = 16; o; o >>= 1) {
                    mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
                    mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
                }
            if (lane == 0)
                for (int a = 0; a < 3; ++a) {
                    atomicMin(&d_ord[6 * b0 + a], mn[a]);
                    atomicMax(&d_ord[6 * b0 + 3 + a], mx[a]);
                }
        } else if (ok) {
            for (int a = 0; a < 3; ++a) {
                atomicMin(&d_ord[6 * b + a], mn[a]);
                atomicMax(&d_ord[6 * b + 3 + a], mx[a]);
            }
        }
    }
}

// One network: every thread folds its elements into a running min / max, then the
// block reduces (warp shuffles, then shared memory) and issues six atomics, instead
// of six per warp and grid stride.
__global__ void __launch_bounds__(256) bbox_one_kernel(const float *__restrict__ x,
                                                       const float *__restrict__ y,
                                                       const float *__restrict__ z, int64_t n,
                                                       uint32_t *d_ord)
{
    __shared__ uint32_t s_red[8][6];
    uint32_t v[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float p[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (p[a] == p[a]) {
                const uint32_t o = ordered(p[a]);
                v[a] = min(v[a], o);
                v[3 + a] = max(v[3 + a], o);
            }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o; o >>= 1) {
            v[a] = min(v[a], __shfl_xor_sync(0xffffffffu, v[a], o));
            v[3 + a] = max(v[3 + a], __shfl_xor_sync(0xffffffffu, v[3 + a], o));
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 6; ++a) s_red[w][a] = v[a];
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        uint32_t r = s_red[0][a];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
            r = a < 3 ? min(r, s_red[k][a]) : max(r, s_red[k][a]);
        if (a < 3)
            atomicMin(&d_ord[a], r);
        else
            atomicMax(&d_ord[a], r);
    }
}

// Also writes the offsets {0, n} of a single network when off_one is given.
__global__ void bbox_init_kernel(uint32_t *d_ord, int32_t B, int64_t *off_one, int64_t n)
{
    if (off_one && blockIdx.x == 0 && threadIdx.x == 0) {
        off_one[0] = 0;
        off_one[1] = n;
    }
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 6 * (int64_t)B;
         k += (int64_t)gridDim.x * blockDim.x)
        d_ord[k] = (k % 6) < 3 ? 0xffffffffu : 0u;
}

struct Box {
    float lo[3], hi[3];
    int given;
};

// Domain box, FP32 inverse extents (IEEE division, as the quantisation formula
// states) and the longest edge in FP64.
// The fixed-point frame of the bottom-up sums covers the box and every position:
// origin = min(box lo, position min), 2^k chosen so that the largest span is
// below 2^30 units.
__global__ void geom_kernel(const uint32_t *d_ord_all, Box box, Geom *g_all, int32_t B)
{
    const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint32_t *d_ord = d_ord_all + 6 * b;
    Geom *g = g_all + b;
    float lo[3], hi[3], blo[3], bhi[3];
    for (int a = 0; a < 3; ++a) {
        const bool any = d_ord[a] != 0xffffffffu; // else every coordinate is NaN
        blo[a] = any ? unordered(d_ord[a]) : 0.0f;
        bhi[a] = any ? unordered(d_ord[3 + a]) : 0.0f;
        lo[a] = box.given ? box.lo[a] : blo[a];
        hi[a] = box.given ? box.hi[a] : bhi[a];
    }
    double ext = 0.0, span = 0.0;
    for (int a = 0; a < 3; ++a) {
        g->lo[a] = lo[a];
        g->hi[a] = hi[a];
        float e = __fsub_rn(hi[a], lo[a]);
        g->inv[a] = e > 0.0f ? __fdiv_rn(1.0f, e) : 0.0f;
        double ed = (double)hi[a] - (double)lo[a];
        if (ed > ext) ext = ed;
        const double o = fmin((double)lo[a], (double)blo[a]);
        const double top = fmax((double)hi[a], (double)bhi[a]);
        g->fx_lo[a] = o;
        if (top - o > span) span = top - o;
    }
    g->ext = ext;
    int k = 30;
    if (span > 0.0) k = 29 - ilogb(span); // span * 2^k < 2^30
    k = max(-60, min(k, 60));
    g->fx_scale = ldexp(1.0, k);
    g->fx_inv = ldexp(1.0, -k);
}

__global__ void fixed_pos_kernel(const float4 *__restrict__ pos, int64_t n,
                                 const int32_t *__restrict__ net, const Geom *__restrict__ g_all,
                                 int4 *__restrict__ posq)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const Geom *g = g_all + net_at(net, s);
        const double ox = g->fx_lo[0], oy = g->fx_lo[1], oz = g->fx_lo[2], sc = g->fx_scale;
        const float4 p = pos[s];
        // NaN or out-of-range coordinates become 0 (the cast is defined as saturating)
        posq[s] = make_int4(__double2int_rn(((double)p.x - ox) * sc),
                            __double2int_rn(((double)p.y - oy) * sc),
                            __double2int_rn(((double)p.z - oz) * sc), 0);
    }
}

// Spread the low 10 bits of v to every third bit.
__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t quantise(float x, float lo, float inv)
{
    float t = __fmul_rn(__fmul_rn(__fsub_rn(x, lo), inv), 1024.0f);
    t = fminf(fmaxf(t, 0.0f), 1023.0f); // NaN -> 0
    return __float2uint_rz(t);
}

// 30-bit Morton code of neuron i in its network's domain. One network: codes32;
// several: keys64 = (network << 30) | code, so one sort orders networks, then space.
__global__ void morton_kernel(const float *__restrict__ x, const float *__restrict__ y,
                              const float *__restrict__ z, int64_t n,
                              const int64_t *__restrict__ off, int32_t B,
                              const Geom *__restrict__ g_all, uint32_t *__restrict__ codes32,
                              uint64_t *__restrict__ keys64, int32_t *__restrict__ ids)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = B == 1 ? 0 : net_of(off, B, i);
        const Geom *g = g_all + b;
        uint32_t qx = quantise(x[i], g->lo[0], g->inv[0]), qy = quantise(y[i], g->lo[1], g->inv[1]),
                 qz = quantise(z[i], g->lo[2], g->inv[2]);
        const uint32_t code = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
        if (B == 1)
            codes32[i] = code;
        else
            keys64[i] = ((uint64_t)b << 30) | code;
        ids[i] = (int32_t)i;
    }
}

__global__ void split_keys_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                  uint32_t *__restrict__ codes, int32_t *__restrict__ net)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[s];
        codes[s] = (uint32_t)(k & 0x3fffffffu);
        net[s] = (int32_t)(k >> 30);
    }
}

__global__ void gather_pos_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                  const float *__restrict__ z, const int32_t *__restrict__ perm,
                                  int64_t n, float4 *__restrict__ pos)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = perm[s];
        pos[s] = make_float4(x[i], y[i], z[i], 0.0f);
    }
}

// Number of leading octal digits shared by codes a and b (10 when equal).
__device__ __forceinline__ int common_digits(uint32_t a, uint32_t b)
{
    uint32_t d = a ^ b;
    return d ? (__clz(d) - 2) / 3 : 10;
}

// First index in [lo, hi) with codes[idx] >= key (codes sorted ascending).
__device__ __forceinline__ int64_t lower_bound(const uint32_t *codes, int64_t lo, int64_t hi,
                                               uint32_t key)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (codes[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// First index in [lo, hi) with (codes[idx] >> shift) > prefix.
__device__ __forceinline__ int64_t upper_bound_prefix(const uint32_t *codes, int64_t lo,
                                                      int64_t hi, uint32_t prefix, int shift)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((codes[mid] >> shift) <= prefix)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Each adjacent pair (j, j+1) of one network that first separates two child cells
// of a depth-d cell (d = common digits) marks that cell as a node: bit d of
// mask[cell start]. The first position of every network holds its root (bit 0).
__global__ void topo_pairs_kernel(const uint32_t *__restrict__ codes,
                                  const int32_t *__restrict__ net,
                                  const int64_t *__restrict__ off, int64_t n,
                                  uint32_t *__restrict__ mask)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = net_at(net, j);
        const int64_t lo = off[b];
        if (j == lo) atomicOr(&mask[j], 1u); // the root of network b
        if (j + 1 >= off[b + 1]) continue;    // last neuron of its network: no pair
        const uint32_t cj = codes[j];
        const int d = common_digits(cj, codes[j + 1]);
        int64_t L;
        if (d == kMaxDepth) {
            if (j > lo && codes[j - 1] == cj) continue; // not the first pair of the bucket
            L = j;
        } else {
            const int s1 = 3 * (kMaxDepth - 1 - d); // child cell (depth d + 1) prefix
            const uint32_t key = (cj >> s1) << s1;
            const int64_t Lc = lower_bound(codes, lo, j, key);
            if (Lc > lo && common_digits(codes[Lc - 1], codes[Lc]) >= d) continue;
            L = Lc;
        }
        atomicOr(&mask[L], 1u << d);
    }
}

__global__ void topo_count_kernel(const uint32_t *__restrict__ mask, int64_t n,
                                  int32_t *__restrict__ cnt)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x)
        cnt[i] = i < n ? __popc(mask[i]) + 1 : 0;
}

// Parent of a node whose shallower ancestors do not start at position i: the
// node of depth common_digits(i-1, i) that contains positions i-1 and i.
__device__ __forceinline__ int32_t parent_across(const uint32_t *codes, const uint32_t *mask,
                                                 const int32_t *base, int64_t lo, int64_t i,
                                                 int *pdepth)
{
    int dp = common_digits(codes[i - 1], codes[i]);
    int sh = 3 * (kMaxDepth - dp);
    uint32_t key = dp == 0 ? 0u : ((codes[i] >> sh) << sh);
    int64_t Lp = lower_bound(codes, lo, i, key);
    *pdepth = dp;
    return base[Lp] + __popc(mask[Lp] & ((1u << dp) - 1u));
}

__global__ void topo_emit_kernel(const uint32_t *__restrict__ codes,
                                 const int32_t *__restrict__ net,
                                 const int64_t *__restrict__ off, int64_t n,
                                 const uint32_t *__restrict__ mask,
                                 const int32_t *__restrict__ base, Node *__restrict__ nodes,
                                 int32_t *__restrict__ parent, int32_t *__restrict__ nsize,
                                 int32_t *__restrict__ leaf_of)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t m = mask[i];
        const int32_t b = base[i];
        const uint32_t ci = codes[i];
        const int32_t nb = net_at(net, i);
        const int64_t lo = off[nb], hi = off[nb + 1];
        int rank = 0;
        for (uint32_t mm = m; mm; mm &= mm - 1) {
            int d = __ffs(mm) - 1;
            int32_t v = b + rank;
            int sh = 3 * (kMaxDepth - d);
            int64_t R = d == 0 ? hi - 1 : upper_bound_prefix(codes, i, hi, ci >> sh, sh) - 1;
            int32_t par = -1;
            if (rank > 0) {
                par = v - 1;
            } else if (i > lo) {
                int pd;
                par = parent_across(codes, mask, base, lo, i, &pd);
            }
            Node nd;
            nd.g = NodeGeo{0.f, 0.f, 0.f, 0.f};
            nd.t = NodeTopo{base[R + 1], (uint32_t)d << 24, (int32_t)i, 0};
            nodes[v] = nd;
            parent[v] = par;
            nsize[v] = (int32_t)(R - i + 1);
            ++rank;
        }
        // the leaf of position i
        int32_t v = b + rank;
        int32_t par;
        if (m) {
            par = v - 1; // the deepest node starting at i
        } else {
            int pd;
            par = parent_across(codes, mask, base, lo, i, &pd);
        }
        Node nd;
        nd.g = NodeGeo{0.f, 0.f, 0.f, 0.f};
        nd.t = NodeTopo{v + 1, kLeafShift, (int32_t)i, 0};
        nodes[v] = nd;
        parent[v] = par;
        nsize[v] = 1;
        leaf_of[i] = v;
    }
}

// The root of network b is the first node at its first Morton position; its
// escape index is where the next network's tree starts.
// Network roots; and nodes m .. m + 2 (past the last node, inside the node array)
// as sentinels for walks that step past the end: no count, escape = next node.
__global__ void roots_kernel(const int32_t *__restrict__ base, const int64_t *__restrict__ off,
                             int32_t B, int32_t *__restrict__ root, Node *nodes,
                             const int64_t *d_num_nodes)
{
    const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) root[b] = base[off[b]];
    if (b < 3) {
        const int64_t m = *d_num_nodes + b;
        nodes[m].g = NodeGeo{0.f, 0.f, 0.f, 0.f};
        nodes[m].t = NodeTopo{(int32_t)(m + 1), 0u, -1, 0};
    }
}

// Bottom-up update as prefix sums (Sec. III-B "Division of work": an inner node
// holds the sum of its children's counts and their count-weighted average
// position, i.e. the sums over the neurons of its cell). Neurons of a cell are a
// contiguous Morton range [first, first + size), so with the exclusive prefix P of
// w = (c, c xq, c yq, c zq) over Morton order, a node's sums are
// P[first + size] - P[first]. Positions enter as fixed-point integers
// xq = round((x - origin) * 2^k) < 2^30 (resolution 2^-k, about 1e-5 um for a
// 10 mm domain), so every sum is an exact int64: order-independent, no
// cancellation, and no FP64 in the scan. centroid = origin + (sum / count) * 2^-k.
struct L4 {
    long long c, x, y, z;
};

__device__ __forceinline__ L4 l4_add(L4 a, L4 b) { return L4{a.c + b.c, a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ L4 l4_sub(L4 a, L4 b) { return L4{a.c - b.c, a.x - b.x, a.y - b.y, a.z - b.z}; }

__device__ __forceinline__ L4 l4_shfl_up(L4 v, int o)
{
    return L4{__shfl_up_sync(0xffffffffu, v.c, o), __shfl_up_sync(0xffffffffu, v.x, o),
              __shfl_up_sync(0xffffffffu, v.y, o), __shfl_up_sync(0xffffffffu, v.z, o)};
}

// Inclusive block scan of L4 over NT threads; *total = block sum.
template <int NT = 256>
__device__ __forceinline__ L4 l4_block_inclusive(L4 v, L4 *total)
{
    constexpr int NW = NT / 32;
    __shared__ L4 wt[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        L4 t = l4_shfl_up(v, o);
        if (lane >= o) v = l4_add(v, t);
    }
    if (lane == 31) wt[warp] = v;
    __syncthreads();
    if (warp == 0) {
        L4 w = lane < NW ? wt[lane] : L4{0, 0, 0, 0};
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            L4 t = l4_shfl_up(w, o);
            if (lane >= o) w = l4_add(w, t);
        }
        if (lane < NW) wt[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v = l4_add(v, wt[warp - 1]);
    *total = wt[NW - 1];
    __syncthreads();
    return v;
}

constexpr int kRedItems = 4;
constexpr int kRedTile = 256 * kRedItems;

// The prefix P runs in passes with no waiting between blocks: leaves and tile sums,
// then each tile's prefix (up to kRedDirect tiles each block adds up the tile sums
// before its own; beyond that one block first scans the tile sums).

// Sum of v over a block of 256 threads (every thread receives it).
__device__ __forceinline__ L4 l4_block_sum(L4 v, L4 *wt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1)
        v = l4_add(v, L4{__shfl_xor_sync(0xffffffffu, v.c, o), __shfl_xor_sync(0xffffffffu, v.x, o),
                         __shfl_xor_sync(0xffffffffu, v.y, o),
                         __shfl_xor_sync(0xffffffffu, v.z, o)});
    if (lane == 0) wt[warp] = v;
    __syncthreads();
    L4 t{0, 0, 0, 0};
#pragma unroll
    for (int w = 0; w < 8; ++w) t = l4_add(t, wt[w]);
    __syncthreads();
    return t;
}

// Pass 1: the leaf nodes of tile t (whole 32-byte nodes; consecutive threads on
// consecutive Morton positions) and the tile's sum of w.
__global__ void __launch_bounds__(256)
    reduce_leaves_kernel(Node *__restrict__ nodes, const int32_t *__restrict__ leaf_of,
                         const int32_t *__restrict__ perm, const float4 *__restrict__ pos,
                         const int4 *__restrict__ posq, const int32_t *__restrict__ vac_de,
                         int64_t n, L4 *__restrict__ tile_sum)
{
    __shared__ L4 s_part[8];
    const int64_t tile0 = (int64_t)blockIdx.x * kRedTile;
    L4 acc{0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < kRedItems; ++k) {
        const int64_t s = tile0 + k * 256 + threadIdx.x;
        if (s < n) {
            int32_t c = vac_de[perm[s]];
            if (c < 0) c = 0;
            const float4 p = pos[s];
            const int32_t v = leaf_of[s];
            Node nd;
            nd.g = c > 0 ? NodeGeo{p.x, p.y, p.z, (float)c} : NodeGeo{0.f, 0.f, 0.f, 0.f};
            nd.t = NodeTopo{v + 1, kLeafShift, (int32_t)s, c};
            nodes[v] = nd;
            const int4 q = posq[s];
            const long long lc = c;
            acc = l4_add(acc, L4{lc, lc * q.x, lc * q.y, lc * q.z});
        }
    }
    const L4 tot = l4_block_sum(acc, s_part);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// Pass 2 (one block of 1024 threads): tile sums -> exclusive tile prefixes, in place;
// P[n] = the total.
__global__ void __launch_bounds__(1024)
    reduce_tiles_kernel(L4 *__restrict__ tile_sum, int64_t nb, L4 *__restrict__ P, int64_t n)
{
    const int64_t per = (nb + 1023) / 1024;
    const int64_t j0 = min((int64_t)threadIdx.x * per, nb), j1 = min(j0 + per, nb);
    L4 acc{0, 0, 0, 0};
    for (int64_t j = j0; j < j1; ++j) acc = l4_add(acc, tile_sum[j]);
    L4 tot;
    L4 run = l4_sub(l4_block_inclusive<1024>(acc, &tot), acc);
    for (int64_t j = j0; j < j1; ++j) {
        const L4 w = tile_sum[j];
        tile_sum[j] = run;
        run = l4_add(run, w);
    }
    if (threadIdx.x == 0) P[n] = tot;
}

// Pass 3: P over tile t = the tile's prefix + the exclusive scan of w inside the tile
// (thread i: positions 4i .. 4i + 3 of the tile). direct: tile holds the tile sums
// and each block adds up those before its own (at most kRedDirect tiles: no pass 2,
// and the last block writes P[n]); else tile holds the prefixes pass 2 formed.
constexpr int64_t kRedDirect = 2048;
__global__ void __launch_bounds__(256)
    reduce_prefix_kernel(const int32_t *__restrict__ perm, const int4 *__restrict__ posq,
                         const int32_t *__restrict__ vac_de, int64_t n,
                         const L4 *__restrict__ tile, L4 *__restrict__ P, bool direct)
{
    __shared__ L4 s_part[8];
    L4 pre{0, 0, 0, 0};
    if (direct) {
        for (int64_t j = threadIdx.x; j < (int64_t)blockIdx.x; j += 256)
            pre = l4_add(pre, tile[j]);
        pre = l4_block_sum(pre, s_part);
    } else {
        pre = tile[blockIdx.x];
    }
    const int64_t s0 = (int64_t)blockIdx.x * kRedTile + (int64_t)threadIdx.x * kRedItems;
    L4 w[kRedItems];
    L4 acc{0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < kRedItems; ++k) {
        const int64_t s = s0 + k;
        w[k] = L4{0, 0, 0, 0};
        if (s < n) {
            int32_t c = vac_de[perm[s]];
            if (c < 0) c = 0;
            const int4 q = posq[s];
            const long long lc = c;
            w[k] = L4{lc, lc * q.x, lc * q.y, lc * q.z};
        }
        acc = l4_add(acc, w[k]);
    }
    L4 tot;
    L4 run = l4_add(pre, l4_sub(l4_block_inclusive(acc, &tot), acc));
#pragma unroll
    for (int k = 0; k < kRedItems; ++k) {
        if (s0 + k < n) P[s0 + k] = run;
        run = l4_add(run, w[k]);
    }
    if (direct && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) P[n] = l4_add(pre, tot);
}

// a + b = s + e exactly (Knuth's two-sum, any magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// r (|r| < 2^43) as hi + lo, both exact floats: hi the multiple of 2^21, lo the rest.
__device__ __forceinline__ void split21(int64_t r, float &hi, float &lo)
{
    hi = __fmul_rn(__int2float_rn((int32_t)(r >> 21)), 2097152.0f);
    lo = __uint2float_rn((uint32_t)(r & 0x1FFFFF));
}

// One centroid coordinate: the float nearest to o + (s / c) * scale for the exact
// fixed-point sum 0 <= s <= (2^30 - 1) c, the count 1 <= c < 2^31 = cf + cl (cf the
// float nearest to c, cl the exact rest), rc = 1 / cf rounded, and scale = 2^-k, all
// in FP32 and integer arithmetic (GB300 runs about two FP64 lanes per clock per SM).
// The quotient: an FP32 estimate q of s / c, corrected twice by the exact integer
// remainder r = s - q c until -c <= r < 2c; then r / c as an unevaluated pair fh + fl
// (fh = r * rc, fl from the exact residual r - fh c), relative error about 2^-44.
// The coordinate: o + q scale + (fh + fl) scale summed with error-free two-sums (the
// products by the power of two are exact) and rounded once.
__device__ __forceinline__ float centroid_coord(int64_t s, int64_t c, float cf, float cl, float rc,
                                                float o, float scale)
{
    const float sf = __fmaf_rn(__uint2float_rn((uint32_t)(s >> 32)), 4294967296.0f,
                               __uint2float_rn((uint32_t)s));
    int64_t q = (int64_t)__float2uint_rz(__fmul_rn(sf, rc)); // within 2^9 of s / c
    int64_t r = s - q * c;
    float rh, rl;
    split21(r, rh, rl);
    q += __float2int_rd(__fmul_rn(__fadd_rn(rh, rl), rc)); // floor(s / c), or one off
    r = s - q * c;                                         // -c <= r < 2c
    split21(r, rh, rl);
    float rf, rerr;
    two_sum(rh, rl, rf, rerr); // r = rf + rerr exactly
    const float fh = __fmul_rn(rf, rc);
    float e = __fmaf_rn(-fh, cf, rf); // rf - fh cf, exact
    e = __fsub_rn(__fadd_rn(e, rerr), __fmul_rn(fh, cl));
    const float fl = __fmul_rn(e, rc);
    const float qa = __int2float_rn((int32_t)(q & ~(int64_t)0xFFFF)); // exact
    const float qb = __int2float_rn((int32_t)(q & 0xFFFF));           // exact
    float h1, e1, h2, e2, h3, e3;
    two_sum(o, __fmul_rn(qa, scale), h1, e1);
    two_sum(h1, __fmul_rn(qb, scale), h2, e2);
    two_sum(h2, __fmul_rn(fh, scale), h3, e3);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), e3), __fmul_rn(fl, scale));
    return __fadd_rn(h3, lo);
}

__device__ __forceinline__ void inner_sums(Node *__restrict__ nodes, int64_t v, int64_t first,
                                           int64_t size, const L4 *__restrict__ P,
                                           const Geom *g)
{
    const L4 s = l4_sub(P[first + size], P[first]);
    if (s.c > 0) {
        // origin and unit are floats exactly (a float corner; a power of two)
        const float scale = (float)g->fx_inv;
        const float cf = __uint2float_rn((uint32_t)s.c);
        const float cl = __int2float_rn((int32_t)(s.c - (int64_t)__float2uint_rn(cf)));
        const float rc = __frcp_rn(cf);
        nodes[v].g = NodeGeo{centroid_coord(s.x, s.c, cf, cl, rc, (float)g->fx_lo[0], scale),
                             centroid_coord(s.y, s.c, cf, cl, rc, (float)g->fx_lo[1], scale),
                             centroid_coord(s.z, s.c, cf, cl, rc, (float)g->fx_lo[2], scale),
                             (float)s.c};
    } else {
        nodes[v].g = NodeGeo{0.f, 0.f, 0.f, 0.f};
    }
    nodes[v].t.icount = (int32_t)s.c;
}

// Inner nodes: exact sums from the prefix, centroid rounded once to FP32. Every inner
// node but a network root holds at least two neurons, so nodes with nsize < 2 (the
// leaves, written by reduce_leaves_kernel) are passed over without reading them;
// thread b < B handles network b's root if it sits above a single leaf.
__global__ void reduce_nodes_kernel(Node *__restrict__ nodes, const int32_t *__restrict__ nsize,
                                    const int64_t *d_num_nodes, const L4 *__restrict__ P,
                                    const int32_t *__restrict__ net,
                                    const Geom *__restrict__ g_all,
                                    const int32_t *__restrict__ root,
                                    const int64_t *__restrict__ off, int32_t B, int64_t n)
{
    const int64_t m = *d_num_nodes;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid < B) {
        const int32_t v = B > 1 ? root[tid] : 0;
        const int64_t first = B > 1 ? off[tid] : 0, last = B > 1 ? off[tid + 1] : n;
        if (last - first < 2 && !node_is_leaf(nodes[v].t.shift)) // a root above one leaf
            inner_sums(nodes, v, first, last - first, P, g_all + tid);
    }
    for (int64_t v = tid; v < m; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t size = nsize[v];
        if (size < 2) continue;
        const int32_t first = nodes[v].t.neuron;
        inner_sums(nodes, v, first, size, P, g_all + net_at(net, first));
    }
}

} // namespace

// B networks, network b = neurons off[b] .. off[b + 1] - 1, each non-empty. B > 1:
// c->d_off already holds the offsets (copied on st); B == 1: one network of n
// neurons, whose box may be given.
cudaError_t octree_build(relearn_ctx *c, int64_t n, int32_t B, const float *x, const float *y,
                         const float *z, const float *box_lo, const float *box_hi,
                         cudaStream_t st)
{
    cudaError_t e;
    Box box{};
    box.given = B == 1 && box_lo && box_hi;
    if (box.given)
        for (int a = 0; a < 3; ++a) {
            box.lo[a] = box_lo[a];
            box.hi[a] = box_hi[a];
        }
    const unsigned gn = grid_for(n, 256, c->num_sms);
    const unsigned gb = (unsigned)((B + 255) / 256);
    bbox_init_kernel<<<gb, 256, 0, st>>>(c->d_ord, B, B == 1 ? c->d_off : nullptr, n);
    note_launch();
    if (B == 1)
        bbox_one_kernel<<<gn, 256, 0, st>>>(x, y, z, n, c->d_ord);
    else
        bbox_kernel<<<gn, 256, 0, st>>>(x, y, z, n, c->d_off, B, c->d_ord);
    note_launch();
    geom_kernel<<<gb, 256, 0, st>>>(c->d_ord, box, c->d_geom, B);
    note_launch();
    morton_kernel<<<gn, 256, 0, st>>>(x, y, z, n, c->d_off, B, c->d_geom, c->d_codes, c->d_nkey,
                                      c->d_perm);
    note_launch();
    int which = 0;
    if (B == 1) {
        if ((e = radix_sort_u32(c->d_codes, c->d_codes_alt, c->d_perm, c->d_perm_alt, n, nullptr,
                                30, c->sort, st, &which)))
            return e;
        if (which) { // keep the sorted result in the primary buffers
            if ((e = cudaMemcpyAsync(c->d_codes, c->d_codes_alt, n * sizeof(uint32_t),
                                     cudaMemcpyDeviceToDevice, st)))
                return e;
            if ((e = cudaMemcpyAsync(c->d_perm, c->d_perm_alt, n * sizeof(int32_t),
                                     cudaMemcpyDeviceToDevice, st)))
                return e;
        }
    } else {
        int bits = 1;
        while (bits < 31 && (1ll << bits) < B) ++bits;
        if ((e = radix_sort_u64(c->d_nkey, c->d_nkey_alt, c->d_perm, c->d_perm_alt, n, nullptr,
                                30 + bits, c->sort, st, &which)))
            return e;
        if (which && (e = cudaMemcpyAsync(c->d_perm, c->d_perm_alt, n * sizeof(int32_t),
                                          cudaMemcpyDeviceToDevice, st)))
            return e;
        split_keys_kernel<<<gn, 256, 0, st>>>(which ? c->d_nkey_alt : c->d_nkey, n, c->d_codes,
                                              c->d_net);
        note_launch();
    }
    int32_t *net = B > 1 ? c->d_net : nullptr;
    gather_pos_kernel<<<gn, 256, 0, st>>>(x, y, z, c->d_perm, n, c->d_pos);
    note_launch();
    fixed_pos_kernel<<<gn, 256, 0, st>>>(c->d_pos, n, net, c->d_geom, c->d_posq);
    note_launch();
    if ((e = cudaMemsetAsync(c->d_mask, 0, n * sizeof(uint32_t), st))) return e;
    topo_pairs_kernel<<<gn, 256, 0, st>>>(c->d_codes, net, c->d_off, n, c->d_mask);
    note_launch();
    topo_count_kernel<<<grid_for(n + 1, 256, c->num_sms), 256, 0, st>>>(c->d_mask, n, c->d_cnt);
    note_launch();
    if ((e = scan_exclusive(c->d_cnt, c->d_base, n + 1, nullptr, c->d_i64 + I64_NODES, c->scan,
                            st)))
        return e;
    topo_emit_kernel<<<gn, 256, 0, st>>>(c->d_codes, net, c->d_off, n, c->d_mask, c->d_base,
                                         c->d_nodes, c->d_parent, c->d_nsize, c->d_leaf);
    note_launch();
    roots_kernel<<<gb, 256, 0, st>>>(c->d_base, c->d_off, B, c->d_root, c->d_nodes,
                                     c->d_i64 + I64_NODES);
    note_launch();
    return cudaGetLastError();
}

cudaError_t octree_reduce(relearn_ctx *c, const int32_t *vac_de, cudaStream_t st)
{
    const int64_t n = c->n;
    const int64_t nb = (n + kRedTile - 1) / kRedTile;
    L4 *P = reinterpret_cast<L4 *>(c->d_acc); // n + 1 prefix entries
    L4 *tile = P + (n + 1);                     // nb tile sums, then tile prefixes
    if (nb > 0) {
        reduce_leaves_kernel<<<(unsigned)nb, 256, 0, st>>>(c->d_nodes, c->d_leaf, c->d_perm,
                                                            c->d_pos, c->d_posq, vac_de, n, tile);
        note_launch();
    }
    // up to kRedDirect tiles each prefix block adds up the tile sums before it itself
    const bool direct = nb > 0 && nb <= kRedDirect;
    if (!direct) {
        reduce_tiles_kernel<<<1, 1024, 0, st>>>(tile, nb, P, n);
        note_launch();
    }
    if (nb > 0) {
        reduce_prefix_kernel<<<(unsigned)nb, 256, 0, st>>>(c->d_perm, c->d_posq, vac_de, n, tile,
                                                            P, direct);
        note_launch();
    }
    reduce_nodes_kernel<<<grid_for(c->max_nodes, 256, c->num_sms), 256, 0, st>>>(
        c->d_nodes, c->d_nsize, c->d_i64 + I64_NODES, P, c->num_nets > 1 ? c->d_net : nullptr,
        c->d_geom, c->d_root, c->d_off, c->num_nets, n);
    note_launch();
    return cudaGetLastError();
}

} // namespace rl

// ---------------------------------------------------------------------------
// Allocation-free Morton ordering: relearn_morton_order_noalloc (relearn.h).
//
// Some callers cannot call cudaMalloc at the point where they need the spatial
// order of their neurons: code running inside another framework's memory pool
// or allocator hooks, real-time loops that must not block on the driver's
// allocator, or plug-ins that only receive already-allocated buffers. This
// entry point serves them: the caller passes the positions and the two output
// arrays, and the sort's scratch (ping-pong buffers, digit histograms, scan
// sums, box words) lives in one file-scope device array instead of a context.
//
// The array is sized for kNoAllocMaxN neurons (about 8.5 MB); every GPU that
// loads this library keeps it until the process exits. All calls on a device
// share it and it keeps the previous call's contents, so calls whose GPU work
// overlaps (different streams, no ordering between them) race on it. Nothing in
// it has to start at zero except the box words, which every call resets, and the
// scans' tile states, which start at zero (static storage) and which every scan
// clears again when it finishes.
// ---------------------------------------------------------------------------
namespace rl {
namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 20;
constexpr int64_t kNoAllocSortBlocks = (kNoAllocMaxN + 2047) / 2048;     // 2048 keys per tile
constexpr int64_t kNoAllocScanBlocks = 1024;                             // >= hist scan tiles
constexpr size_t kOffGeom = 256;
constexpr size_t kOffCodesAlt = 512;
constexpr size_t kOffPermAlt = kOffCodesAlt + 4 * size_t(kNoAllocMaxN);
constexpr size_t kOffHist = kOffPermAlt + 4 * size_t(kNoAllocMaxN);
constexpr size_t kOffScan = kOffHist + 4 * 256 * size_t(kNoAllocSortBlocks);
constexpr size_t kOffScanFlags = kOffScan + 8 * 2 * size_t(kNoAllocScanBlocks);
constexpr size_t kOffStatus = kOffScanFlags + 4 * size_t(kNoAllocScanBlocks + 3);
constexpr size_t kNoAllocBytes = kOffStatus + 4;
// the regions must not overlap: the box words (6 x uint32) below the geometry, the
// geometry below the sort's ping-pong buffers; 8-byte sums on 8-byte boundaries
static_assert(6 * sizeof(uint32_t) <= kOffGeom, "box words overlap the geometry");
static_assert(kOffGeom + sizeof(Geom) <= kOffCodesAlt, "geometry overlaps the sort buffers");
static_assert(kOffHist % 8 == 0 && kOffScan % 8 == 0, "scan sums must be 8-byte aligned");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
    unsigned char *base = nullptr; // device address of g_noalloc_scratch on this device
    int num_sms = 0;
};
std::mutex g_noalloc_mu;
int g_noalloc_sms[64]; // SM count per device ordinal, read once

// With the device current: the array's device address (looked up on every call, so
// that a context re-created after cudaDeviceReset is served with its own address)
// and the SM count (read once per device).
relearn_status noalloc_setup(int dev, NoAllocDevice *out)
{
    if (dev < 0 || dev >= 64) return RELEARN_ERR_INVALID_ARG;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
        return RELEARN_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_sms[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return RELEARN_ERR_CUDA;
        g_noalloc_sms[dev] = sms > 0 ? sms : 1;
    }
    out->base = static_cast<unsigned char *>(p);
    out->num_sms = g_noalloc_sms[dev];
    return RELEARN_OK;
}

} // namespace

} // namespace rl

extern "C" relearn_status relearn_morton_order_noalloc(int64_t n, const float *x, const float *y,
                                                       const float *z, const float *box_lo3,
                                                       const float *box_hi3, uint32_t *codes,
                                                       int32_t *perm, void *stream)
{
    using namespace rl;
    if (n < 1 || !x || !y || !z || !codes || !perm) return RELEARN_ERR_INVALID_ARG;
    if ((box_lo3 == nullptr) != (box_hi3 == nullptr)) return RELEARN_ERR_INVALID_ARG;
    if (box_lo3)
        for (int a = 0; a < 3; ++a)
            if (!(box_hi3[a] >= box_lo3[a])) return RELEARN_ERR_INVALID_ARG;
    if (n > kNoAllocMaxN) return RELEARN_ERR_CAPACITY;
    if (sort_blocks_needed(n) > kNoAllocSortBlocks ||
        scan_blocks_needed(256 * sort_blocks_needed(n)) > kNoAllocScanBlocks)
        return RELEARN_ERR_CAPACITY;
    // a launch error left pending by earlier work belongs to its owner: refuse the call
    // and leave it pending, so that the checks below see this call's launches only
    if (cudaPeekAtLastError() != cudaSuccess) return RELEARN_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RELEARN_ERR_CUDA;
    NoAllocDevice d;
    relearn_status s = noalloc_setup(dev, &d);
    if (s != RELEARN_OK) return s;
    uint32_t *ord = reinterpret_cast<uint32_t *>(d.base);
    Geom *geom = reinterpret_cast<Geom *>(d.base + kOffGeom);
    uint32_t *codes_alt = reinterpret_cast<uint32_t *>(d.base + kOffCodesAlt);
    int32_t *perm_alt = reinterpret_cast<int32_t *>(d.base + kOffPermAlt);
    SortScratch ss;
    ss.hist = reinterpret_cast<int32_t *>(d.base + kOffHist);
    ss.max_blocks = kNoAllocSortBlocks;
    ss.scan.block_sums = reinterpret_cast<int64_t *>(d.base + kOffScan);
    ss.scan.flags = reinterpret_cast<int32_t *>(d.base + kOffScanFlags);
    // a scan wait that runs out (it cannot: every wait ends) would be recorded here
    ss.scan.status = reinterpret_cast<int32_t *>(d.base + kOffStatus);
    ss.scan.max_blocks = kNoAllocScanBlocks;
    cudaStream_t st = (cudaStream_t)stream;
    Box box{};
    box.given = box_lo3 != nullptr;
    if (box.given)
        for (int a = 0; a < 3; ++a) {
            box.lo[a] = box_lo3[a];
            box.hi[a] = box_hi3[a];
        }
    const unsigned grid = grid_for(n, 256, d.num_sms);
    // One network: the box and Morton kernels never read the network offsets.
    bbox_init_kernel<<<1, 32, 0, st>>>(ord, 1, nullptr, n); // geom_kernel reads the box
    note_launch();
    bbox_one_kernel<<<grid, 256, 0, st>>>(x, y, z, n, ord);
    note_launch();
    geom_kernel<<<1, 1, 0, st>>>(ord, box, geom, 1);
    note_launch();
    morton_kernel<<<grid, 256, 0, st>>>(x, y, z, n, nullptr, 1, geom, codes, nullptr, perm);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return RELEARN_ERR_CUDA;
    int which = 0;
    if (radix_sort_u32(codes, codes_alt, perm, perm_alt, n, nullptr, 30, ss, st, &which) !=
        cudaSuccess)
        return RELEARN_ERR_CUDA;
    if (which) {
        if (cudaMemcpyAsync(codes, codes_alt, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess ||
            cudaMemcpyAsync(perm, perm_alt, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
            return RELEARN_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? RELEARN_OK : RELEARN_ERR_CUDA;
}

