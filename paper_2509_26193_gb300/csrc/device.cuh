// Device-side helpers shared by the library's kernels (not by the oracle).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rl {

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplies
// with the Weyl key schedule. Written from the published definition.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t lo0 = m0 * c.x, hi0 = __umulhi(m0, c.x);
        uint32_t lo1 = m1 * c.z, hi1 = __umulhi(m1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t philox_x(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                             uint64_t seed)
{
    return philox4x32_10(make_uint4(w0, w1, w2, w3),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)))
        .x;
}

// 2^x on the special-function unit (PTX ex2.approx, flush-to-zero).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt(x) and 1 / x on the special-function unit (PTX sqrt.approx and rcp.approx,
// flush-to-zero): a relative error of a few 2^-24, far inside the differentiable
// form's tolerances, for one instruction instead of a correctly rounded sequence.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// First error wins; the host reads it on the next synchronising call.
__device__ __forceinline__ void set_status(int32_t *status, int32_t code)
{
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// One octree node, 32 bytes (one L2 sector): geometry refreshed by every
// bottom-up update, topology fixed by the build.
struct __align__(16) NodeGeo {
    float cx, cy, cz; // count-weighted centroid (0 when count == 0)
    float cnt;        // vacant dendritic elements, as float
};
struct __align__(16) NodeTopo {
    int32_t escape;  // pre-order index just past this node's subtree
    uint32_t shift;  // inner node of depth d: d << 24; leaf: kLeafShift (see below)
    int32_t neuron;  // leaves: Morton position of the neuron; inner: first position
    int32_t icount;  // vacant dendritic elements, exact
};
struct __align__(32) Node {
    NodeGeo g;
    NodeTopo t;
};

// A whole node (32 bytes, 32-byte aligned) in one 256-bit read-only load
// (PTX ld.global.nc.v8.f32, sm_100 and later): geometry and escape/shift.
__device__ __forceinline__ void load_node(const Node *n, float4 &g, int2 &t)
{
    float v[8];
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
          "=f"(v[7])
        : "l"(n));
    g = make_float4(v[0], v[1], v[2], v[3]);
    t = make_int2(__float_as_int(v[4]), __float_as_int(v[5]));
}

constexpr int kMaxDepth = 10;


// Number of leading octal digits (octree levels) two Morton codes share; 10 when equal.
__device__ __forceinline__ int morton_common_digits(uint32_t a, uint32_t b)
{
    const uint32_t d = a ^ b;
    return d ? (__clz(d) - 2) / 3 : 10;
}

// The acceptance test of a node at depth d, d^2 > thr0 / 4^d, is evaluated as
// d^2 * 4^d > thr0 by adding d << 24 to the bits of d^2 (2d to its exponent;
// exact, as is the division of thr0 by 4^d), and comparing the result as an
// unsigned integer with the bits of thr0 (positive floats order like their
// bits). A leaf gets a shift so large that the sum always exceeds any finite
// thr0: single neurons are always accepted.
constexpr uint32_t kLeafShift = 0x7F800000u;
__host__ __device__ __forceinline__ bool node_is_leaf(uint32_t shift) { return shift == kLeafShift; }
__host__ __device__ __forceinline__ int depth_of(uint32_t shift) { return (int)(shift >> 24); }

} // namespace rl
