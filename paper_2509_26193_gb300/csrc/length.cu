// Differentiable form (not in the paper): the expected synapse length over each
// source's root frontier and its adjoint.
//
// For a source i with m_i = vac_ax[i] > 0, its root frontier F_i is the set of
// candidates of its first draw (Sec. III-B search from the root, criterion of
// Sec. II), its own leaf excluded. With D_ik = |x_i - c_k|^2, d_ik = sqrt(D_ik),
// a_ik = N_k exp(-D_ik / sigma^2), S_i = sum_k a_ik and q_ik = a_ik / S_i:
//   l_i = sum_k q_ik d_ik,   L = sum_i m_i l_i / M,   M = sum of m_i with S_i > 0.
// Adjoint (criterion and topology constant):
//   dl_i/dsigma = (2 / sigma^3) sum_k q_ik (d_ik - l_i) (D_ik - Dbar_i),
//   dl_i/dc_k   = q_ik r_ik (2 (d_ik - l_i) / sigma^2 - 1 / d_ik),  r = x_i - c_k,
//   dl_i/dx_i   = -sum_k dl_i/dc_k,   dc_k/dx_j = w_j / N_k  (w = vac_de).
//
// Forward: one walk of each root frontier (the search kernel's warp-union walk: the
// warp's 32 sources, cut at the boundaries of depth-5 cells, depth 4 in the adjoint,
// walk one union per piece), FP32 attractions with Kahan-compensated sums; S, l and
// Dbar formed in FP64 and kept per source with the exponent shift. Backward: the
// same walk again,
// recomputing every attraction (nothing per candidate is stored), accumulating
// the centroid adjoints G_k = sum_i (m_i / M) dl_i/dc_k per node in FP64 and each
// source's direct term in registers (Kahan-compensated FP32: it is a sum of terms of
// both signs that nearly cancel); then every neuron j adds w_j * sum over its cells
// k of G_k / N_k (its leaf's parent chain, in FP64).
//
// Node adjoints: in a union walk every lane that takes a candidate takes the same
// node at the same step, so the warp first sums its lanes' (x, y, z) contributions
// (a transpose reduction: five shuffle levels that leave each component's total on
// eight lanes) and three lanes add the totals to the node with FP64 atomics; a warp
// cut into pieces does this once per piece that took a candidate. One FP32 vector
// atomic per lane and candidate (the previous design) was L2-atomic-bound and its
// order-dependent FP32 sums left element-wise gradient errors up to 6e-3 of the
// cancellation-aware scale at 2^18 neurons; FP64 sums of warp partials bring every
// element within the FP32 arithmetic of its terms.
#include "internal.h"

namespace rl {

namespace {

constexpr float kTinyL = 8.673617e-19f; // 2^-60: below this S is redone with a shift
// Sources in one cell this deep share a walk. The forward pass cuts finer: its
// pieces step in blocks like one union, so more pieces cost little (2^18 cube,
// forward: depth 4 2.11 ms, 5 1.77 ms, 6 2.02 ms). The adjoint sums every piece's
// contributions across the warp at each step, so more pieces cost a warp sum each
// (adjoint: depth 4 5.77 ms, 5 10.8 ms, 6 31.0 ms).
constexpr int kFwdDepth = 5, kBwdDepth = 4;
constexpr int kLenBlock = 128; // walk steps between progress checks

struct LenArgs {
    const Node *__restrict__ nodes;
    const float4 *__restrict__ pos;
    const int32_t *__restrict__ perm;
    const int32_t *__restrict__ act_src;
    const uint32_t *__restrict__ codes;
    const int32_t *__restrict__ leaf_of;
    const int32_t *__restrict__ vac_ax;
    const int64_t *d_total; // active sources
    int64_t *evals_total;   // candidates visited (both passes)
    const SearchConst *sc;
    float4 *state;  // [n] per Morton position
    double *lsum;   // [4]
    int32_t *work;
    // backward
    double *G;           // [4 * nodes] centroid adjoints (x, y, z, unused) in FP64
    float *gx, *gy, *gz; // id order
    const double *gout;  // upstream gradient of the mean (NULL = 1)
    double *gsigma;
};

__device__ __forceinline__ float att(float cnt, float D, float k2, float k2sh)
{
    return __fmul_rn(cnt, ex2_approx(__fmaf_rn(-k2, D, k2sh)));
}

__device__ __forceinline__ void kahan(float &sum, float &c, float a)
{
    const float y = __fsub_rn(a, c);
    const float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

struct Fwd {
    float s = 0.f, sc = 0.f, a = 0.f, ac = 0.f, b = 0.f, bc = 0.f;
    float dmin2 = __builtin_huge_valf();
};

struct Bwd {
    float cov = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    float cx = 0.f, cy = 0.f, cz = 0.f; // Kahan compensation of the direct term
};

struct Src {
    float3 x;
    int32_t self;
    float l, Db, invS, k2sh, w; // backward: state and (m_i gout / M)
};

// One candidate (accepted, count > 0, not the source's own leaf).
__device__ __forceinline__ void fwd_visit(Fwd &f, float cnt, float D, float k2, float k2sh)
{
    const float at = att(cnt, D, k2, k2sh);
    const float d = sqrt_approx(D);
    kahan(f.s, f.sc, at);
    kahan(f.a, f.ac, __fmul_rn(at, d));
    kahan(f.b, f.bc, __fmul_rn(at, D));
    f.dmin2 = fminf(f.dmin2, D);
}

// Returns the node's adjoint contribution (m_i / M) dl_i/dc_k in (ox, oy, oz).
__device__ __forceinline__ void bwd_visit(Bwd &b, const Src &s, float cnt, float rx, float ry,
                                          float rz, float D, float k2, float two_s2, float &ox,
                                          float &oy, float &oz)
{
    const float q = __fmul_rn(att(cnt, D, k2, s.k2sh), s.invS);
    const float d = sqrt_approx(D);
    const float dl = __fsub_rn(d, s.l);
    b.cov = __fmaf_rn(__fmul_rn(q, dl), __fsub_rn(D, s.Db), b.cov);
    const float inv_d = d > 0.0f ? rcp_approx(d) : 0.0f;
    const float kap = __fmul_rn(__fmul_rn(q, __fmaf_rn(two_s2, dl, -inv_d)), s.w);
    ox = __fmul_rn(kap, rx);
    oy = __fmul_rn(kap, ry);
    oz = __fmul_rn(kap, rz);
    kahan(b.gx, b.cx, -ox);
    kahan(b.gy, b.cy, -oy);
    kahan(b.gz, b.cz, -oz);
}

// One lane's own contribution straight to the node (lane-by-lane walks, rare).
__device__ __forceinline__ void add_node(double *G, int32_t p, float ox, float oy, float oz)
{
    atomicAdd(&G[4 * (int64_t)p + 0], (double)ox);
    atomicAdd(&G[4 * (int64_t)p + 1], (double)oy);
    atomicAdd(&G[4 * (int64_t)p + 2], (double)oz);
}

// Sum of (x, y, z) over the 32 lanes (every lane calls it). Transpose reduction: at
// offset 16 a lane keeps two of the four values (x, y, z, 0) and sends the other
// two; at offset 8 it keeps one; offsets 4, 2, 1 sum that one. Afterwards lanes
// 0-7 hold the total of x, 8-15 of y, 16-23 of z. Returns this lane's total.
__device__ __forceinline__ float warp_sum3(float x, float y, float z, int lane)
{
    const bool hi = lane & 16;
    float k0 = hi ? z : x, k1 = hi ? 0.0f : y;
    const float s0 = hi ? x : z, s1 = hi ? y : 0.0f;
    k0 = __fadd_rn(k0, __shfl_xor_sync(0xffffffffu, s0, 16));
    k1 = __fadd_rn(k1, __shfl_xor_sync(0xffffffffu, s1, 16));
    const bool b3 = lane & 8;
    float k = b3 ? k1 : k0;
    k = __fadd_rn(k, __shfl_xor_sync(0xffffffffu, b3 ? k0 : k1, 8));
    k = __fadd_rn(k, __shfl_xor_sync(0xffffffffu, k, 4));
    k = __fadd_rn(k, __shfl_xor_sync(0xffffffffu, k, 2));
    k = __fadd_rn(k, __shfl_xor_sync(0xffffffffu, k, 1));
    return k;
}

// The warp's contributions to node p (every lane calls it with the same p; lanes
// that took no candidate pass zeros): summed across the warp, then added to the
// node's FP64 adjoint by lanes 0, 8 and 16 (x, y, z).
__device__ __forceinline__ void add_node_warp(double *G, int32_t p, float ox, float oy, float oz,
                                              int lane)
{
    const float t = warp_sum3(ox, oy, oz, lane);
    if ((lane & 7) == 0 && lane < 24) atomicAdd(&G[4 * (int64_t)p + (lane >> 3)], (double)t);
}

// A lane's own walk of its root frontier (stackless: expand = p + 1, accept or
// empty = escape).
template <bool kBack>
__device__ int32_t lane_walk(const LenArgs &a, const Src &s, int32_t end, uint32_t thr0, float k2,
                             float k2sh, float two_s2, Fwd &f, Bwd &b)
{
    int32_t p = 1, visited = 0;
    while (p < end) {
        const float4 g = __ldg(reinterpret_cast<const float4 *>(&a.nodes[p].g));
        const int2 t = __ldg(reinterpret_cast<const int2 *>(&a.nodes[p].t));
        const float rx = __fsub_rn(s.x.x, g.x), ry = __fsub_rn(s.x.y, g.y),
                    rz = __fsub_rn(s.x.z, g.z);
        const float D = __fmaf_rn(rx, rx, __fmaf_rn(ry, ry, __fmul_rn(rz, rz)));
        const bool has = g.w > 0.0f;
        const bool pass = __float_as_uint(D) + (uint32_t)t.y > thr0;
        if (has && pass && p != s.self) {
            ++visited;
            if constexpr (!kBack) {
                fwd_visit(f, g.w, D, k2, k2sh);
            } else {
                float ox, oy, oz;
                bwd_visit(b, s, g.w, rx, ry, rz, D, k2, two_s2, ox, oy, oz);
                add_node(a.G, p, ox, oy, oz);
            }
        }
        p = (has && !pass) ? p + 1 : max(t.x, p + 1);
    }
    return visited;
}

#ifndef RELEARN_LEN_BWD_MIN_BLOCKS
#define RELEARN_LEN_BWD_MIN_BLOCKS 5 // the adjoint's warp sums need more than 40 registers
#endif
// The forward pass at 6 blocks per SM (its three compensated sums need the
// registers: 8 blocks took the 2^18-neuron forward pass from 2.46 to 3.08 ms), the
// adjoint at 5 (6 blocks: 6.08 -> 6.32 ms).
template <bool kBack>
__global__ void __launch_bounds__(256, kBack ? RELEARN_LEN_BWD_MIN_BLOCKS : 6)
    length_kernel(LenArgs a)
{
    const int32_t A = (int32_t)*a.d_total;
    const int lane = threadIdx.x & 31;
    const uint32_t thr0 = __ldg(&a.sc->thr0);
    const float k2 = __ldg(&a.sc->k2);
    const float sigma = __ldg(&a.sc->sigma);
    const float two_s2 = (float)(2.0 / ((double)sigma * (double)sigma));
    const int32_t root_end = __ldg(&a.nodes[0].t.escape);
    double wscale = 0.0;
    if constexpr (kBack) {
        const double M = a.lsum[1];
        wscale = M > 0.0 ? (a.gout ? *a.gout : 1.0) / M : 0.0;
    }
    double my0 = 0.0, my1 = 0.0;
    int64_t my_evals = 0;
    for (;;) {
        int32_t nb = 0;
        if (lane == 0) nb = atomicAdd(a.work, 32);
        nb = __shfl_sync(0xffffffffu, nb, 0);
        if (nb >= A) break;
        const int32_t slot = nb + lane;
        const bool live = slot < A;
        const int32_t sp = live ? a.act_src[slot] : -1;
        Src s;
        const float4 xp = live ? a.pos[sp] : make_float4(0.f, 0.f, 0.f, 0.f);
        s.x = make_float3(xp.x, xp.y, xp.z);
        s.self = live ? a.leaf_of[sp] : -1;
        const int32_t i = live ? a.perm[sp] : 0;
        s.l = s.Db = s.invS = s.k2sh = s.w = 0.0f;
        bool on_src = live; // takes part as a source (backward: included in M)
        if constexpr (kBack) {
            if (live) {
                const float4 st = a.state[sp];
                s.l = st.x;
                s.Db = st.y;
                s.invS = st.z;
                s.k2sh = st.w;
            }
            on_src = live && s.invS > 0.0f;
            s.w = on_src ? (float)((double)a.vac_ax[i] * wscale) : 0.0f;
        }
        // the 32 sources (Morton order) are cut wherever two neighbours do not share a
        // cell of depth kFwdDepth (kBwdDepth); each piece walks one union (one piece: uni)
        const int last = min(A - 1 - nb, 31);
        uint32_t code = live ? a.codes[sp] : 0u;
        code = __shfl_sync(0xffffffffu, code, live ? lane : last);
        const uint32_t nxt = __shfl_down_sync(0xffffffffu, code, 1);
        const uint32_t cuts = __ballot_sync(
            0xffffffffu,
            lane < 31 && morton_common_digits(code, nxt) < (kBack ? kBwdDepth : kFwdDepth));
        const bool uni = cuts == 0;
        Fwd f;
        Bwd b;
        // The walks step in blocks of four steps per bounds test: nodes root_end ..
        // root_end + 2 are sentinels (no count, escape = the next node), and a piece
        // whose walk has ended parks on root_end (its escape clamped back to it).
        // Escapes are taken as stored; each block of kLenBlock steps must advance,
        // which keeps a walk over a malformed tree finite.
        int32_t p = 1, skip = on_src ? 0 : 0x7fffffff;
        if (!uni) {
            const uint32_t below = cuts & ((1u << lane) - 1u);
            const int first = below ? 32 - __clz(below) : 0;
            const uint32_t from = cuts >> lane;
            const int lastl = from ? lane + __ffs(from) - 1 : 31;
            const uint32_t gmask = (lastl == 31 ? 0xffffffffu : ((1u << (lastl + 1)) - 1u)) &
                                   ~((1u << first) - 1u);
            auto piece_step = [&]() {
                float4 g;
                int2 t;
                load_node(&a.nodes[p], g, t); // one 256-bit read
                const float rx = __fsub_rn(s.x.x, g.x), ry = __fsub_rn(s.x.y, g.y),
                            rz = __fsub_rn(s.x.z, g.z);
                const float D = __fmaf_rn(rx, rx, __fmaf_rn(ry, ry, __fmul_rn(rz, rz)));
                const bool on = p >= skip && g.w > 0.0f;
                const bool pass = __float_as_uint(D) + (uint32_t)t.y > thr0;
                const bool take = on && pass && p != s.self;
                if (on && pass) skip = t.x;
                my_evals += take ? 1 : 0;
                if constexpr (!kBack) {
                    if (take) fwd_visit(f, g.w, D, k2, 0.0f);
                } else {
                    float ox = 0.0f, oy = 0.0f, oz = 0.0f;
                    if (take) bwd_visit(b, s, g.w, rx, ry, rz, D, k2, two_s2, ox, oy, oz);
                    // one warp sum per piece that took a candidate at this step
                    const uint32_t took = __ballot_sync(0xffffffffu, take) & gmask;
                    uint32_t heads = __ballot_sync(0xffffffffu, lane == first && took != 0u);
                    while (heads) {
                        const int h = __ffs(heads) - 1;
                        heads &= heads - 1;
                        const bool mine = first == h;
                        add_node_warp(a.G, __shfl_sync(0xffffffffu, p, h), mine ? ox : 0.0f,
                                      mine ? oy : 0.0f, mine ? oz : 0.0f, lane);
                    }
                }
                const uint32_t down = __ballot_sync(0xffffffffu, on && !pass) & gmask;
                p = min(down ? p + 1 : t.x, root_end);
            };
            while (__any_sync(0xffffffffu, p < root_end)) {
                const int32_t p_blk = p;
                int k = 0;
#pragma unroll 1
                for (; k < kLenBlock && __any_sync(0xffffffffu, p < root_end); k += 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) piece_step();
                }
                if (__any_sync(0xffffffffu, p < root_end && p <= p_blk)) break;
            }
        } else {
            auto uni_step = [&]() {
                float4 g;
                int2 t;
                load_node(&a.nodes[p], g, t); // one 256-bit read
                const float rx = __fsub_rn(s.x.x, g.x), ry = __fsub_rn(s.x.y, g.y),
                            rz = __fsub_rn(s.x.z, g.z);
                const float D = __fmaf_rn(rx, rx, __fmaf_rn(ry, ry, __fmul_rn(rz, rz)));
                const bool on = p >= skip && g.w > 0.0f;
                const bool pass = __float_as_uint(D) + (uint32_t)t.y > thr0;
                const bool take = on && pass && p != s.self;
                if (on && pass) skip = t.x;
                my_evals += take ? 1 : 0;
                if constexpr (!kBack) {
                    if (take) fwd_visit(f, g.w, D, k2, 0.0f);
                } else {
                    float ox = 0.0f, oy = 0.0f, oz = 0.0f;
                    if (take) bwd_visit(b, s, g.w, rx, ry, rz, D, k2, two_s2, ox, oy, oz);
                    if (__any_sync(0xffffffffu, take)) add_node_warp(a.G, p, ox, oy, oz, lane);
                }
                p = __any_sync(0xffffffffu, on && !pass) ? p + 1 : t.x;
            };
            while (p < root_end) {
                const int32_t p_blk = p;
#pragma unroll 1
                for (int k = 0; k < kLenBlock && p < root_end; k += 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) uni_step();
                }
                if (p <= p_blk) break;
            }
        }
        if constexpr (!kBack) {
            if (!live) continue;
            double S = (double)f.s - (double)f.sc;
            float k2sh = 0.0f;
            if (S < (double)kTinyL && f.dmin2 < __int_as_float(0x7f800000)) {
                // every term underflowed: redo with the exponents shifted by the nearest D
                k2sh = __fmul_rn(k2, f.dmin2);
                f = Fwd();
                Bwd unused;
                my_evals += lane_walk<false>(a, s, root_end, thr0, k2, k2sh, two_s2, f, unused);
                S = (double)f.s - (double)f.sc;
            }
            float4 st = make_float4(0.f, 0.f, 0.f, k2sh);
            if (S > 0.0) {
                const double l = ((double)f.a - (double)f.ac) / S;
                st.x = (float)l;
                st.y = (float)(((double)f.b - (double)f.bc) / S);
                st.z = (float)(1.0 / S);
                const double m = (double)a.vac_ax[i];
                my0 += m * l;
                my1 += m;
            }
            a.state[sp] = st;
        } else {
            if (!on_src) continue;
            a.gx[i] = __fsub_rn(b.gx, b.cx);
            a.gy[i] = __fsub_rn(b.gy, b.cy);
            a.gz[i] = __fsub_rn(b.gz, b.cz);
            my0 += (double)s.w * (double)b.cov; // * 2 / sigma^3 below
        }
    }
    for (int o = 16; o; o >>= 1) {
        my0 += __shfl_xor_sync(0xffffffffu, my0, o);
        my1 += __shfl_xor_sync(0xffffffffu, my1, o);
        my_evals += __shfl_xor_sync(0xffffffffu, my_evals, o);
    }
    if (lane == 0 && my_evals)
        atomicAdd(reinterpret_cast<unsigned long long *>(a.evals_total),
                  (unsigned long long)my_evals);
    if (lane == 0) {
        if constexpr (!kBack) {
            if (my1 > 0.0) {
                atomicAdd(&a.lsum[0], my0);
                atomicAdd(&a.lsum[1], my1);
            }
        } else if (a.gsigma && my0 != 0.0) {
            const double sd = (double)sigma;
            atomicAdd(a.gsigma, my0 * 2.0 / (sd * sd * sd));
        }
    }
}

// Active sources (vac_ax > 0) in Morton order.
__global__ void len_flags_kernel(const int32_t *__restrict__ vac_ax,
                                 const int32_t *__restrict__ perm, int64_t n,
                                 int32_t *__restrict__ flag)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= n;
         s += (int64_t)gridDim.x * blockDim.x)
        flag[s] = s < n && vac_ax[perm[s]] > 0 ? 1 : 0;
}

__global__ void len_fill_kernel(const int32_t *__restrict__ flag,
                                const int32_t *__restrict__ off, int64_t n,
                                int32_t *__restrict__ act_src)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x)
        if (flag[s]) act_src[off[s]] = (int32_t)s;
}

// mean = sum m l / M (NaN when M = 0); ell[id] = l (NaN for excluded neurons).
__global__ void len_finish_kernel(const float4 *__restrict__ state,
                                  const int32_t *__restrict__ flag,
                                  const int32_t *__restrict__ perm, int64_t n, double *lsum,
                                  float *ell, double *mean)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        const double m = lsum[1] > 0.0 ? lsum[0] / lsum[1] : __longlong_as_double(0x7ff8000000000000LL);
        lsum[2] = m;
        if (mean) *mean = m;
    }
    if (!ell) return;
    for (int64_t s = tid; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const float4 st = state[s];
        ell[perm[s]] = flag[s] && st.z > 0.0f ? st.x : __int_as_float(0x7fc00000);
    }
}

__global__ void zero_nodes_kernel(double4 *G, const int64_t *d_num_nodes)
{
    const int64_t m = *d_num_nodes;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x)
        G[k] = make_double4(0.0, 0.0, 0.0, 0.0);
}

// Neuron j (Morton position s) gets w_j * sum over its cells k of G_k / N_k.
__global__ void len_scatter_kernel(const Node *__restrict__ nodes,
                                   const int32_t *__restrict__ parent,
                                   const int32_t *__restrict__ leaf_of,
                                   const int32_t *__restrict__ perm,
                                   const int32_t *__restrict__ vac_de, const double *__restrict__ G,
                                   int64_t n, float *gx, float *gy, float *gz)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = perm[s];
        const int32_t w = vac_de[i];
        if (w <= 0) continue;
        double hx = 0.0, hy = 0.0, hz = 0.0;
        for (int32_t u = leaf_of[s]; u >= 0; u = parent[u]) {
            const int32_t cnt = nodes[u].t.icount;
            if (cnt <= 0) continue;
            const double inv = 1.0 / (double)cnt;
            hx += G[4 * (int64_t)u + 0] * inv;
            hy += G[4 * (int64_t)u + 1] * inv;
            hz += G[4 * (int64_t)u + 2] * inv;
        }
        // direct term (FP32) + cell terms (FP64), rounded once
        gx[i] = (float)((double)gx[i] + w * hx);
        gy[i] = (float)((double)gy[i] + w * hy);
        gz[i] = (float)((double)gz[i] + w * hz);
    }
}

LenArgs make_args(relearn_ctx *c, const int32_t *vac_ax)
{
    LenArgs a{};
    a.nodes = c->d_nodes;
    a.pos = c->d_pos;
    a.perm = c->d_perm;
    a.act_src = c->d_act_src;
    a.codes = c->d_codes;
    a.leaf_of = c->d_leaf;
    a.vac_ax = vac_ax;
    a.d_total = c->d_i64 + I64_ACTIVE;
    a.evals_total = c->d_i64 + I64_LEN_EVALS;
    a.sc = c->d_sc;
    a.state = c->d_lstate;
    a.lsum = c->d_lsum;
    a.work = c->d_i32 + I32_WORK;
    return a;
}

template <bool kBack>
cudaError_t launch_length(relearn_ctx *c, const LenArgs &a, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->d_i32 + I32_WORK, 0, sizeof(int32_t), st))) return e;
    void (*kern)(LenArgs) = length_kernel<kBack>;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0))) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<c->num_sms * per_sm, 256, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

} // namespace

cudaError_t length_forward(relearn_ctx *c, const int32_t *vac_ax, float *ell, double *mean,
                           cudaStream_t st)
{
    cudaError_t e;
    const int64_t n = c->n;
    int32_t *flag = c->d_cnt;
    len_flags_kernel<<<grid_for(n + 1, 256, c->num_sms), 256, 0, st>>>(vac_ax, c->d_perm, n,
                                                                        flag);
    note_launch();
    if ((e = scan_exclusive(flag, c->d_act_off, n + 1, nullptr, c->d_i64 + I64_ACTIVE, c->scan,
                            st)))
        return e;
    len_fill_kernel<<<grid_for(n, 256, c->num_sms), 256, 0, st>>>(flag, c->d_act_off, n,
                                                                   c->d_act_src);
    note_launch();
    if ((e = cudaMemsetAsync(c->d_lsum, 0, 4 * sizeof(double), st))) return e;
    if ((e = launch_length<false>(c, make_args(c, vac_ax), st))) return e;
    len_finish_kernel<<<grid_for(n, 256, c->num_sms), 256, 0, st>>>(c->d_lstate, flag,
                                                                     c->d_perm, n, c->d_lsum,
                                                                     ell, mean);
    note_launch();
    return cudaGetLastError();
}

cudaError_t length_backward(relearn_ctx *c, const int32_t *vac_ax, const int32_t *vac_de,
                            const double *grad_mean, float *gx, float *gy, float *gz,
                            double *gsigma, cudaStream_t st)
{
    cudaError_t e;
    const int64_t n = c->n;
    // d_acc is free between bottom-up updates (32 bytes per node: x, y, z in FP64)
    double *G = c->d_acc;
    zero_nodes_kernel<<<grid_for(c->max_nodes, 256, c->num_sms), 256, 0, st>>>(
        reinterpret_cast<double4 *>(G), c->d_i64 + I64_NODES);
    note_launch();
    for (float *g : {gx, gy, gz})
        if ((e = cudaMemsetAsync(g, 0, n * sizeof(float), st))) return e;
    if (gsigma && (e = cudaMemsetAsync(gsigma, 0, sizeof(double), st))) return e;
    LenArgs a = make_args(c, vac_ax);
    a.G = G;
    a.gx = gx;
    a.gy = gy;
    a.gz = gz;
    a.gout = grad_mean;
    a.gsigma = gsigma;
    if ((e = launch_length<true>(c, a, st))) return e;
    len_scatter_kernel<<<grid_for(n, 256, c->num_sms), 256, 0, st>>>(
        c->d_nodes, c->d_parent, c->d_leaf, c->d_perm, vac_de, G, n, gx, gy, gz);
    note_launch();
    return cudaGetLastError();
}

} // namespace rl
