// Barnes-Hut partner search (Sec. III-B "Division of work", second paragraph;
// acceptance criterion and theta from Sec. II).
//
// Work item = one source neuron with vacant axonal elements. All searches of a
// neuron start at the root from the same position, so their root frontier and
// its total attraction S are identical; only the Philox draw differs. The root
// frontier is therefore evaluated once per neuron and each of the neuron's
// searches then draws from it (results are exactly those of separate searches).
//
// Root pass (pass 1): the 32 lanes of a warp take 32 neurons that are adjacent
// in Morton order and walk the UNION of their frontiers together (or, when they
// straddle a cell boundary, one union per piece). Nodes are in pre-order with
// skip links, so the walk is stackless: the warp descends (p + 1) if any lane
// rejects the node under the acceptance criterion, else jumps to the node's
// escape index. A lane that accepted a node ignores the node's subtree; every
// node is loaded once per union (one broadcast load), and each lane still meets
// exactly its own candidates in Morton order, which is the order of the
// cumulative draw. Every kCkStride union steps each lane stores a checkpoint
// (its next own node, its running sum); when the list is full, every other
// checkpoint is dropped and checkpoints are stored half as often, so a draw never
// walks more than one interval however long the walk.
//
// Updates with few sources run bh_split_kernel instead (one warp per source, its
// frontier walk shared out among the lanes; see there).
//
// Sums: each lane accumulates its own terms in FP32 with Kahan compensation (the
// running total is sum - c, accurate to a few ulp whatever the number of terms);
// S, the root-level normaliser, is formed in FP64 from (sum, c).
//
// Draw (pass 2): u * S is located between two checkpoints by binary search and the
// lane walks its own candidates from there, repeating pass 1's compensated
// arithmetic bit for bit (explicit round-to-nearest intrinsics), until its running
// total exceeds u * S. An inner node that is drawn restarts the search from itself;
// restart frontiers are small and are walked per lane (sum, then find).
//
// Attraction a = count * 2^(-k2 d^2 + k2sh), k2 = log2(e) / sigma^2. k2sh = 0
// unless every term would underflow, in which case the pass is redone with the
// exponents shifted by the nearest candidate's d^2 (an exact common factor).
#include <cooperative_groups.h>

#include "internal.h"
#include "scan_pair.cuh"

namespace rl {

namespace {

constexpr int kCkStride = 128; // warp steps between checkpoints (times 2^k once the list fills)
constexpr int kMaxCk = 128;    // checkpoints kept per lane
constexpr float kTiny = 8.673617e-19f; // 2^-60
// Walks per warp (see bh_search_kernel): the warp's 32 sources are cut into pieces at
// the boundaries of cells of some depth, and each piece walks one union. With one
// network the warp's pieces step in blocks of four like a single union, so fine cuts
// cost little: depth kCutSingle (cells of 1/64 of the domain's edge). Sweep on the
// 2^20-neuron clustered network (first three updates, 86 / 40 / 15 % of the neurons
// searching): depth 2 6.85 / 4.12 / 2.74 ms, depth 4 6.87 / 3.78 / 2.27, depth 5
// 6.83 / 3.78 / 2.16, depth 6 6.77 / 3.78 / 2.16, depth 7 7.24 / 4.10 / 2.81,
// depth 10 13.65 / 6.84 / 4.05. With several networks (pieces stepped one step per
// test) the cut follows the share of neurons searching: the more search, the closer
// consecutive sources are, and the coarser the cut can be before a union spans
// sources too far apart: depth 2 when at least kDenseTenths / 10 of the neurons
// search, depth 3 from kMidTenths / 10, else depth 4 (a batch of 256 uniform
// networks, 86 % searching: depth 2 234.9 ms, depth 4 274.2 ms).
constexpr int kCutSingle = 6;
constexpr int kCutDense = 2, kCutMid = 3, kCutSparse = 4, kDenseTenths = 6, kMidTenths = 3;
// The default also looks at how many sources the update has, per resident warp of
// the union kernel (W = 9,728 on 152 SMs at 8 blocks per SM; the sweeps below were
// taken at 6 blocks, W = 7,296, and the threshold rechecked at 8). Per-update sweeps
// on the 2^20-neuron clustered network (ten successive updates, 907k down to 2.4k
// sources): with at most kSplitWaves * W sources the split kernel (one warp per
// source) wins (61.8k sources: 1.67 ms against 1.84 ms; 162k: 4.73 ms against
// 2.46 ms), on small trees as well (4096-neuron cube, 4096 sources: 0.10 ms against
// 0.46 ms).
constexpr int kSplitWaves = 9;

// A node of depth d is accepted iff d^2 > thr0 / 4^d, thr0 = (root length / theta)^2
// rounded to FP32 (see NodeTopo::shift). theta = 0 accepts no inner node.
// Network b's constants; per-network sigma/theta replace the scalars when given.
__device__ __forceinline__ void search_const_one(int32_t b, const Geom *g_all, float sigma,
                                                 float theta, const float *net_sigma,
                                                 const float *net_theta, SearchConst *sc_all,
                                                 int32_t *status)
{
    float sg = net_sigma ? net_sigma[b] : sigma;
    float tt = net_theta ? net_theta[b] : theta;
    if (!(sg > 0.0f && sg < 3.0e38f && tt >= 0.0f && tt < 3.0e38f)) {
        set_status(status, RELEARN_ERR_INVALID_ARG); // the update applies nothing
        sg = 1.0f;
        tt = 0.0f;
    }
    const double ext = g_all[b].ext, th = (double)tt;
    const float thr0 = th > 0.0 ? (float)((ext / th) * (ext / th)) : 3.4028234663852886e38f;
    SearchConst *sc = sc_all + b;
    sc->thr0 = __float_as_uint(fminf(thr0, 3.4028234663852886e38f));
    const double s = (double)sg;
    sc->k2 = (float)(1.4426950408889634 / (s * s));
    sc->sigma = sg;
    sc->pad = 0.0f;
}

// One thread per network.
__global__ void search_const_kernel(const Geom *g_all, int32_t B, float sigma, float theta,
                                    const float *net_sigma, const float *net_theta,
                                    SearchConst *sc_all, int32_t *status)
{
    const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) search_const_one(b, g_all, sigma, theta, net_sigma, net_theta, sc_all, status);
}

// The query setup of an update in one pass (a pair scan, scan_pair.cuh): over index
// k < n, a = 1 if the neuron at Morton position k has vacant axonal elements, b = the
// number of searches of neuron id k (canonical request order is by id). Their
// exclusive prefixes place the sources (act_src, Morton order) and the request records
// (id order, qoff_o); thread i < B of the grid also forms network i's search
// constants. Q = total searches; beyond capacity the update is void (status
// CAPACITY), and so it is while an earlier device error (e.g. a bad per-network
// parameter) is unread: finish() publishes Q and the source count only then.
struct QueryOp {
    const int32_t *__restrict__ vac_ax;
    const int32_t *__restrict__ perm;
    int64_t n, max_searches;
    int32_t *__restrict__ qoff_o;
    int32_t *__restrict__ act_src;
    int32_t *__restrict__ req_src;
    int32_t *__restrict__ req_elem;
    int32_t *__restrict__ req_tgt;
    int64_t *d_total, *d_active; // totals of the pass
    int32_t *d_Q, *d_A;          // what the search and the acceptance read
    int64_t *d_Qout, *d_Qsum;    // Q of this update, searches of every update
    int32_t *status;
    // search constants
    const Geom *g_all;
    int32_t B;
    float sigma, theta;
    const float *net_sigma, *net_theta;
    SearchConst *sc_all;

    __device__ void prologue(int64_t i, int64_t stride) const
    {
        for (int64_t b = i; b < B; b += stride)
            search_const_one((int32_t)b, g_all, sigma, theta, net_sigma, net_theta, sc_all,
                             status);
    }
    __device__ int2 load(int64_t k) const
    {
        const int32_t c = vac_ax[k];
        return make_int2(vac_ax[perm[k]] > 0 ? 1 : 0, c > 0 ? c : 0);
    }
    __device__ void emit(int64_t k, int64_t a, int64_t q, int2 v) const
    {
        qoff_o[k] = (int32_t)q;
        if (v.x) act_src[a] = (int32_t)k;
        // requests past the capacity are not written (the update is then void)
        for (int32_t e = 0; e < v.y && q + e < max_searches; ++e) {
            req_src[q + e] = (int32_t)k;
            req_elem[q + e] = e;
            req_tgt[q + e] = -1;
        }
    }
    __device__ void store_totals(int64_t a, int64_t q) const
    {
        *d_active = a;
        *d_total = q;
        qoff_o[n] = (int32_t)q;
    }
    __device__ void finish() const
    {
        const int64_t q = *(volatile int64_t *)d_total;
        const bool over = q > max_searches;
        if (over) set_status(status, RELEARN_ERR_CAPACITY);
        const bool void_ = over || *(volatile int32_t *)status != 0;
        *d_Qout = q;
        *d_Q = void_ ? 0 : (int32_t)q;
        *d_A = void_ ? 0 : (int32_t)*(volatile int64_t *)d_active;
        *d_Qsum += void_ ? 0 : q;
    }
};

struct SearchArgs {
    const Node *__restrict__ nodes;
    const float4 *__restrict__ pos;
    const int32_t *__restrict__ perm;
    const int32_t *__restrict__ act_src;
    const uint32_t *__restrict__ codes;
    const int32_t *__restrict__ leaf_of;
    const int32_t *__restrict__ vac_ax;
    const int32_t *__restrict__ qoff_o;
    const int32_t *d_A;
    const SearchConst *sc; // [networks]
    const int32_t *net;    // network of each Morton position, NULL for one network
    const int32_t *root;   // root node of each network
    int32_t *work;
    int32_t *req_tgt;
    int64_t *failed;
    int64_t *evals_total;
    int64_t *steps_total;
    int count; // add evaluations and walk steps to the totals (RELEARN_FLAG_COUNT or DIAG)
    double *diag_lns;
    int32_t *diag_evals;
    int32_t *diag_restarts;
    uint64_t seed;
    uint32_t step;
    int forced_group; // 0 = choose per warp; 1, 8, 16, 32 = union width; 2 = split
    int spread_depth;  // cut depth of union pieces (-1: the default by source density)
    int64_t n_total;   // neurons of all networks
    int32_t split_below; // with forced_group 0: split kernel for at most this many sources
    int split_cap;       // ranges per source in the split kernel (split_capacity)
    // deferred restarts (RELEARN_FLAG_REGROUP): searches whose first draw is an inner
    // node are queued here and finished after a sort by that node (subtree order)
    int defer;
    const int32_t *req_elem;
    uint32_t *rq_key; // drawn node
    int32_t *rq_val;  // queue slot
    int32_t *rq_out;  // [slot] request index
    int32_t *rq_src;  // [slot] Morton position of the source
    int32_t *rq_count;
};

// Which of the two search kernels serves this launch (both read the same counts).
__device__ __forceinline__ bool split_launch(const SearchArgs &a, int32_t A)
{
    return a.forced_group == 2 ||
           (a.forced_group == 0 && A <= a.split_below);
}

struct WalkOut {
    float sum;
    float dmin2;
    int32_t pick;
    int32_t evals;
};

// Attraction of one candidate; shared by every pass so the sums agree bit for bit.
__device__ __forceinline__ float attraction(float cnt, float d2, float k2, float k2sh)
{
    return __fmul_rn(cnt, ex2_approx(__fmaf_rn(-k2, d2, k2sh)));
}

// d^2 = dx^2 + dy^2 + dz^2 with (dx, dy) as one packed pair (f32x2 subtract and
// multiply, sm_100 and later): one instruction fewer than three scalar lanes. Every
// pass of the search uses this function, so their sums agree bit for bit.
__device__ __forceinline__ float dist2(float3 x, float4 g)
{
    unsigned long long xy, gxy, dxy, sq;
    asm("mov.b64 %0, {%1, %2};" : "=l"(xy) : "f"(x.x), "f"(x.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(gxy) : "f"(g.x), "f"(g.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dxy) : "l"(xy), "l"(gxy));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(sq) : "l"(dxy));
    float sx, sy;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(sx), "=f"(sy) : "l"(sq));
    const float dz = __fsub_rn(x.z, g.z);
    return __fadd_rn(__fmaf_rn(dz, dz, sx), sy);
}

// One lane's own walk over [p0, end) starting from running sum cum0: visits
// exactly its candidates (expand = p + 1, accept or empty = escape).
// FIND = false: total attraction, nearest d^2, evaluations.
// FIND = true: first candidate whose running sum exceeds `target` (else the
// last one with weight, or -1).
template <bool FIND>
__device__ __forceinline__ WalkOut walk(const Node *__restrict__ nodes, int32_t p0, int32_t end,
                                        float cum0, float3 x, int32_t self_node, uint32_t thr0,
                                        float k2, float k2sh, float target)
{
    WalkOut o{0.0f, __int_as_float(0x7f800000), -1, 0};
    int32_t p = p0;
    float cum = cum0;
    while (p < end) {
        float4 g;
        int2 t;
        load_node(&nodes[p], g, t);
        const float d2 = dist2(x, g);
        const bool has = g.w > 0.0f;
        const bool acc = has && (__float_as_uint(d2) + (uint32_t)t.y > thr0);
        const bool take = acc && p != self_node;
        if (!FIND) o.evals += has ? 1 : 0;
        if (take) {
            const float a = attraction(g.w, d2, k2, k2sh);
            cum = __fadd_rn(cum, a);
            if (FIND) {
                if (a > 0.0f) o.pick = p;
                if (cum > target) return o;
            } else {
                o.dmin2 = fminf(o.dmin2, d2);
            }
        }
        // t.x > p holds for every well-formed node; max() keeps the walk finite regardless
        p = (has && !acc) ? p + 1 : max(t.x, p + 1);
    }
    o.sum = cum;
    return o;
}

// One step of a 32-lane union walk at node p (see bh_search_kernel); kCount: count
// this lane's evaluations in own.
template <bool kCount>
__device__ __forceinline__ void union_step(const Node *__restrict__ nodes, int32_t &p,
                                           int32_t &skip, float &cum, float &comp,
                                           int32_t &own, float3 x, int32_t self_node,
                                           uint32_t thr0, float k2, float k2sh);

// Kahan step: sum + a with the rounding error carried in c (explicit round-to-
// nearest operations, so every pass reproduces the same bits).
__device__ __forceinline__ void kahan_add(float &sum, float &c, float a)
{
    const float y = __fsub_rn(a, c);
    const float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

template <bool kCount>
__device__ __forceinline__ void union_step(const Node *__restrict__ nodes, int32_t &p,
                                           int32_t &skip, float &cum, float &comp,
                                           int32_t &own, float3 x, int32_t self_node,
                                           uint32_t thr0, float k2, float k2sh)
{
    float4 g;
    int2 t;
    load_node(&nodes[p], g, t);
    const float d2 = dist2(x, g);
    const bool on = p >= skip && g.w > 0.0f;
    const bool pass = __float_as_uint(d2) + (uint32_t)t.y > thr0;
    if (kCount) own += on ? 1 : 0;
    if (on && pass) {
        skip = t.x;
        if (p != self_node) kahan_add(cum, comp, attraction(g.w, d2, k2, k2sh));
    }
    // escapes lie past their node in every well-formed tree; the caller checks that each
    // block of steps advances, which keeps the walk finite regardless
    p = __any_sync(0xffffffffu, on && !pass) ? p + 1 : t.x;
}

// One step of several union walks in one warp (lane groups gmask; see
// bh_search_kernel): a group whose walk has ended sits on the sentinel node at
// root_end, which has no count, and its escape is clamped back to root_end.
template <bool kCount>
__device__ __forceinline__ void group_step(const Node *__restrict__ nodes, int32_t &p,
                                           int32_t &skip, float &cum, float &comp,
                                           int32_t &own, int32_t &gst, float3 x,
                                           int32_t self_node, uint32_t thr0, float k2,
                                           float k2sh, uint32_t gmask, int32_t root_end)
{
    float4 g;
    int2 t;
    if (kCount) gst += p < root_end ? 1 : 0;
    load_node(&nodes[p], g, t);
    const float d2 = dist2(x, g);
    const bool on = p >= skip && g.w > 0.0f;
    const bool pass = __float_as_uint(d2) + (uint32_t)t.y > thr0;
    if (kCount) own += on ? 1 : 0;
    if (on && pass) {
        skip = t.x;
        if (p != self_node) kahan_add(cum, comp, attraction(g.w, d2, k2, k2sh));
    }
    const uint32_t down = __ballot_sync(0xffffffffu, on && !pass) & gmask;
    p = min(down ? p + 1 : t.x, root_end);
}

// Draw on the root frontier from a checkpoint: the lane's own walk with pass 1's
// compensated arithmetic; returns the first candidate whose running total
// (sum - c) exceeds target, else the last candidate with weight, else -1.
__device__ __forceinline__ int32_t find_root(const Node *__restrict__ nodes, int32_t p,
                                             int32_t end, float cum, float comp, float3 x,
                                             int32_t self_node, uint32_t thr0, float k2,
                                             float k2sh, float target)
{
    int32_t pick = -1;
    while (p < end) {
        float4 g;
        int2 t;
        load_node(&nodes[p], g, t);
        const float d2 = dist2(x, g);
        const bool has = g.w > 0.0f;
        const bool acc = has && (__float_as_uint(d2) + (uint32_t)t.y > thr0);
        if (acc && p != self_node) {
            const float a = attraction(g.w, d2, k2, k2sh);
            kahan_add(cum, comp, a);
            if (a > 0.0f) pick = p;
            if (__fsub_rn(cum, comp) > target) return p;
        }
        p = (has && !acc) ? p + 1 : max(t.x, p + 1);
    }
    return pick;
}

// Restarts after the first draw picked node k: while the drawn node is inner, its
// frontier is walked by this lane (sum, then find), until a leaf is drawn.
// Returns the target neuron (-1: failed); evals and draws count the work.
__device__ __forceinline__ int32_t restart_chain(const SearchArgs &a, int32_t k, float3 x,
                                                  int32_t self_node, uint32_t thr0, float k2,
                                                  int32_t i, int32_t e, int32_t &evals,
                                                  int32_t &draws, int64_t &my_evals)
{
    draws = 1;
    while (k >= 0 && draws < 24) {
        const int4 tk = __ldg(reinterpret_cast<const int4 *>(&a.nodes[k].t));
        if (node_is_leaf((uint32_t)tk.y)) return a.perm[tk.z];
        const int32_t kend = tk.x;
        float sh = 0.0f;
        WalkOut w1 = walk<false>(a.nodes, k + 1, kend, 0.0f, x, self_node, thr0, k2, 0.0f, 0.0f);
        evals += w1.evals;
        my_evals += w1.evals;
        if (w1.sum < kTiny && w1.dmin2 < __int_as_float(0x7f800000)) {
            sh = __fmul_rn(k2, w1.dmin2);
            w1 = walk<false>(a.nodes, k + 1, kend, 0.0f, x, self_node, thr0, k2, sh, 0.0f);
        }
        if (!(w1.sum > 0.0f)) return -1;
        const uint32_t u = philox_x((uint32_t)i, a.step,
                                    ((uint32_t)e << 8) | (uint32_t)depth_of((uint32_t)tk.y), 0u,
                                    a.seed);
        const float target = (float)((double)u * 2.3283064365386963e-10 * (double)w1.sum);
        k = walk<true>(a.nodes, k + 1, kend, 0.0f, x, self_node, thr0, k2, sh, target).pick;
        ++draws;
    }
    return -1;
}

// Keep every other checkpoint (the list is full). Not inlined: it runs at most a few
// times per long walk and keeps its registers out of the walk loop.
__device__ __noinline__ void ck_halve(int32_t *ckp, float *ckc, float *ckk)
{
    for (int j = 0; j < kMaxCk / 2; ++j) {
        ckp[j] = ckp[2 * j];
        ckc[j] = ckc[2 * j];
        ckk[j] = ckk[2 * j];
    }
}

// Deferred restart: queue search `out` of the source at Morton position s with
// its first draw k (warp-aggregated slot allocation).
__device__ __forceinline__ void enqueue_restart(const SearchArgs &a, int32_t k, int32_t out,
                                                int32_t s, double lns0, int32_t evals)
{
    namespace cg = cooperative_groups;
    cg::coalesced_group g = cg::coalesced_threads();
    int32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(a.rq_count, (int32_t)g.size());
    base = g.shfl(base, 0);
    const int32_t slot = base + (int32_t)g.thread_rank();
    a.rq_key[slot] = (uint32_t)k;
    a.rq_val[slot] = slot;
    a.rq_out[slot] = out;
    a.rq_src[slot] = s;
    if (a.diag_lns) {
        a.diag_lns[out] = lns0;
        a.diag_evals[out] = evals;
    }
}

// A warp's sources walk in unions chosen per warp task from where they lie (a union
// is only worth walking when its sources are close: far-apart sources share few
// nodes and most lanes would idle), or in fixed groups of G = 1, 8, 16 or 32 lanes
// when search_group forces a width. A warp runs one walk per union, one node load
// in flight per union and step. Results do not depend on the grouping.
// 8 blocks of 256 threads per SM (32 registers, the most resident warps): the walk
// waits on dependent node reads, and more warps hide more of that latency (first
// update of the clustered benchmark 7.4 ms against 8.1 ms at 6 blocks).
#ifndef RELEARN_SEARCH_MIN_BLOCKS
#define RELEARN_SEARCH_MIN_BLOCKS 8
#endif
// kBatched: several networks, each source walks its own network's tree (root,
// subtree end, threshold and kernel width looked up per work item); else one
// network whose constants are loaded once. kCount: count evaluations and walk steps
// (into the context's totals and the per-search diagnostics); counting costs one
// instruction per union step, so updates that ask for neither skip it.
template <bool kBatched, bool kCount>
__global__ void __launch_bounds__(256, RELEARN_SEARCH_MIN_BLOCKS) bh_search_kernel(SearchArgs a)
{
    const int32_t A = *a.d_A;
    if (split_launch(a, A)) return; // bh_split_kernel serves this launch
    const int lane = threadIdx.x & 31;
    int32_t root = 0, root_end = 0;
    uint32_t thr0 = 0;
    float k2 = 0.0f;
    if constexpr (!kBatched) {
        root_end = __ldg(&a.nodes[0].t.escape);
        thr0 = __ldg(&a.sc->thr0);
        k2 = __ldg(&a.sc->k2);
    }
    int32_t ckp[kMaxCk];
    float ckc[kMaxCk];  // compensated running sum at each checkpoint
    float ckk[kMaxCk];  // its compensation term
    for (;;) {
        int32_t nb = 0;
        if (lane == 0) nb = atomicAdd(a.work, 32);
        nb = __shfl_sync(0xffffffffu, nb, 0);
        if (nb >= A) break;
        const int32_t slot = nb + lane;
        const bool live = slot < A;
        const int32_t s = live ? a.act_src[slot] : -1;
        const float4 xp = live ? a.pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float3 x = make_float3(xp.x, xp.y, xp.z);
        const int32_t self_node = live ? a.leaf_of[s] : -1;
        const int last = min(A - 1 - nb, 31);
        int32_t net = 0, n0 = 0, n31 = 0;
        bool mixed8 = false;
        if constexpr (kBatched) {
            // this lane's network (an idle lane takes the last live lane's): its root,
            // the end of its subtree, its acceptance threshold and kernel width
            net = live ? a.net[s] : 0;
            net = __shfl_sync(0xffffffffu, net, live ? lane : last);
            root = __ldg(&a.root[net]);
            root_end = __ldg(&a.nodes[root].t.escape);
            thr0 = __ldg(&a.sc[net].thr0);
            k2 = __ldg(&a.sc[net].k2);
            n0 = __shfl_sync(0xffffffffu, net, 0);
            n31 = __shfl_sync(0xffffffffu, net, 31);
            const int32_t nf = __shfl_sync(0xffffffffu, net, lane & ~7);
            const int32_t nl = __shfl_sync(0xffffffffu, net, lane | 7);
            mixed8 = __any_sync(0xffffffffu, nf != nl);
        }

        // ---- walks: the warp's 32 sources (Morton order) are cut wherever two
        // neighbours do not share a cell of depth spread_depth (or a network); each
        // piece walks one union. Codes are sorted, so a piece whose neighbours all
        // share that cell lies in one such cell. One piece: a single walk (G = 32).
        int G = a.forced_group;
        uint32_t gmask = 0xffffffffu;
        int seg_first = 0; // first lane of this lane's walk
        if (G == 0) {
            uint32_t code = live ? a.codes[s] : 0u;
            code = __shfl_sync(0xffffffffu, code, live ? lane : last);
            const uint32_t nxt = __shfl_down_sync(0xffffffffu, code, 1);
            const int depth = a.spread_depth >= 0                          ? a.spread_depth
                              : !kBatched                                   ? kCutSingle
                              : (int64_t)A * 10 >= kDenseTenths * a.n_total ? kCutDense
                              : (int64_t)A * 10 >= kMidTenths * a.n_total   ? kCutMid
                                                                            : kCutSparse;
            bool cut = lane < 31 && morton_common_digits(code, nxt) < depth;
            if constexpr (kBatched) {
                const int32_t nn = __shfl_down_sync(0xffffffffu, net, 1);
                cut = cut || (lane < 31 && nn != net);
            }
            const uint32_t cuts = __ballot_sync(0xffffffffu, cut); // bit i: cut after lane i
            const uint32_t below = cuts & ((1u << lane) - 1u);
            seg_first = below ? 32 - __clz(below) : 0;
            const uint32_t from = cuts >> lane;
            const int seg_last = from ? lane + __ffs(from) - 1 : 31;
            gmask = (seg_last == 31 ? 0xffffffffu : ((1u << (seg_last + 1)) - 1u)) &
                    ~((1u << seg_first) - 1u);
            G = cuts ? 0 : 32;
        } else if (kBatched && G > 1 && n0 != n31) {
            // a fixed width whose groups would span networks: the widest that does not
            const int32_t nh = __shfl_sync(0xffffffffu, net, lane & ~15);
            const int32_t nt = __shfl_sync(0xffffffffu, net, lane | 15);
            const bool mixed16 = __any_sync(0xffffffffu, nh != nt);
            G = G == 32 ? (mixed16 ? (mixed8 ? 1 : 8) : 16) : G == 16 && mixed16 ? (mixed8 ? 1 : 8)
                                                                                : G;
            if (G == 8 && mixed8) G = 1;
        }
        if (a.forced_group != 0) {
            gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
            seg_first = lane & ~(G - 1);
        }

        // ---- pass 1: union of the G root frontiers of this lane's group
        float k2sh = 0.0f;
        double S = 0.0; // the root-level normaliser, FP64
        int32_t own = 0, nck = 0, task_steps = 0;
        for (int attempt = 0; attempt < 2; ++attempt) {
            int32_t p = root + 1, skip = live ? 0 : 0x7fffffff, steps = 0;
            float cum = 0.0f, comp = 0.0f; // Kahan sum and compensation
            int32_t ckst = 0; // checkpoints stored (bits 0-7) and log2 of the interval in
                              // blocks (bits 8-15): no further live register in the walk
            own = 0;
            // at the start of each block (`steps` is then a multiple of kCkStride): a
            // checkpoint every 2^(ckst >> 8) blocks; when the list is full keep every other
            // one and store half as often (walks of more than kMaxCk * kCkStride steps)
            auto checkpoint = [&](int32_t at) {
                if (((steps / kCkStride) & ((1 << (ckst >> 8)) - 1)) != 0) return;
                int32_t k = ckst & 0xff;
                if (k == kMaxCk) {
                    ck_halve(ckp, ckc, ckk);
                    k = kMaxCk / 2;
                    ckst += 1 << 8;
                }
                ckp[k] = at;
                ckc[k] = cum;
                ckk[k] = comp;
                ckst = (ckst & ~0xff) | (k + 1);
            };
            if (G == 32) {
                // one walk per warp: every lane steps together, no group masks
                while (p < root_end) {
                    checkpoint(max(p, skip));
                    const int32_t p_blk = p;
                    int k = 0;
                    if constexpr (!kBatched) {
                        // four steps per test: nodes root_end .. root_end + 2 are
                        // sentinels (no count, escape = next node), so steps past the
                        // end change nothing
#pragma unroll 1
                        for (; k < kCkStride && p < root_end; k += 4) {
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                union_step<kCount>(a.nodes, p, skip, cum, comp, own, x,
                                                   self_node, thr0, k2, k2sh);
                        }
                    } else {
#pragma unroll 1
                        for (; k < kCkStride && p < root_end; ++k)
                            union_step<kCount>(a.nodes, p, skip, cum, comp, own, x, self_node,
                                               thr0, k2, k2sh);
                    }
                    steps += k;
                    if (p <= p_blk) break; // no progress: only a malformed tree
                }
                if (p > root_end) steps -= p - root_end; // the sentinels' steps
            } else if constexpr (!kBatched) {
                // several walks per warp (lane groups gmask) in the same blocks of four
                // steps per test: a group that has finished parks on the sentinel at
                // root_end (no count; its escape is clamped back to root_end)
                int32_t gst = 0; // this group's own steps (counted with kCount only)
                while (__any_sync(0xffffffffu, p < root_end)) {
                    if (p < root_end) checkpoint(max(p, skip));
                    const int32_t p_blk = p;
                    int k = 0;
#pragma unroll 1
                    for (; k < kCkStride && __any_sync(0xffffffffu, p < root_end); k += 4) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            group_step<kCount>(a.nodes, p, skip, cum, comp, own, gst, x,
                                               self_node, thr0, k2, k2sh, gmask, root_end);
                    }
                    steps += k;
                    // no progress: only a malformed tree
                    if (__any_sync(0xffffffffu, p < root_end && p <= p_blk)) break;
                }
                steps = gst;
            } else {
                while (__any_sync(0xffffffffu, p < root_end)) {
                    const bool run = p < root_end; // uniform within the group
                    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                    int2 t = make_int2(p + 1, 0);
                    if (run) {
                        if ((steps & (kCkStride - 1)) == 0) checkpoint(max(p, skip));
                        ++steps;
                        load_node(&a.nodes[p], g, t);
                    }
                    const float d2 = dist2(x, g);
                    const bool on = run && p >= skip && g.w > 0.0f;
                    const bool pass = __float_as_uint(d2) + (uint32_t)t.y > thr0;
                    if (kCount) own += on ? 1 : 0;
                    if (on && pass) {
                        skip = t.x;
                        if (p != self_node)
                            kahan_add(cum, comp, attraction(g.w, d2, k2, k2sh));
                    }
                    const uint32_t down = __ballot_sync(0xffffffffu, on && !pass) & gmask;
                    if (run) p = down ? p + 1 : max(t.x, p + 1);
                }
            }
            if (kCount && lane == seg_first) task_steps += steps; // one count per walk
            nck = ckst & 0xff;
            S = (double)cum - (double)comp;
            // every term underflowed: redo with the exponents shifted by the nearest d^2
            const bool redo = live && S < (double)kTiny;
            if (!__any_sync(0xffffffffu, redo)) break;
            if (redo) {
                const WalkOut w = walk<false>(a.nodes, root + 1, root_end, 0.0f, x, self_node,
                                              thr0, k2, k2sh, 0.0f);
                if (w.dmin2 < __int_as_float(0x7f800000)) k2sh = __fmul_rn(k2, w.dmin2);
            }
        }
        int64_t task_evals = own; // 0 on idle lanes (no node is theirs)
        if (live) {
            // ---- draws: every search of this neuron
            const int32_t i = a.perm[s];
            const int32_t nq = max(a.vac_ax[i], 0);
            const int32_t qbase = a.qoff_o[i];
            // ln S for the diagnostics only (an FP64 log per source otherwise wasted)
            const double lns0 = !a.diag_lns ? 0.0
                                : S > 0.0   ? log(S) - (double)k2sh * 0.6931471805599453
                                            : -__longlong_as_double(0x7ff0000000000000LL);
            for (int32_t e = 0; e < nq; ++e) {
                int32_t result = -1, evals = own, draws = 0;
                if (S > 0.0) {
                    uint32_t u = philox_x((uint32_t)i, a.step, (uint32_t)e << 8, 0u, a.seed);
                    const double tgt = (double)u * 2.3283064365386963e-10 * S;
                    // last checkpoint whose running total, formed as the draw walk forms
                    // it (FP32 sum - compensation), does not exceed u * S: the walk from it
                    // never starts past its answer
                    const float ftgt = (float)tgt;
                    int lo = 0, hi = nck - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (__fsub_rn(ckc[mid], ckk[mid]) <= ftgt)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    int32_t k = find_root(a.nodes, ckp[lo], root_end, ckc[lo], ckk[lo], x,
                                          self_node, thr0, k2, k2sh, ftgt);
                    if (k < 0) // u * S rounded up to S past the last weighted candidate
                        k = find_root(a.nodes, root + 1, root_end, 0.0f, 0.0f, x, self_node,
                                      thr0, k2, k2sh, __int_as_float(0x7f800000));
                    if (a.defer && k >= 0 &&
                        !node_is_leaf((uint32_t)__ldg(&a.nodes[k].t.shift))) {
                        enqueue_restart(a, k, qbase + e, s, lns0, evals);
                        continue; // finished by bh_restart_kernel
                    }
                    result = restart_chain(a, k, x, self_node, thr0, k2, i, e, evals, draws,
                                           task_evals);
                }
                const int32_t out = qbase + e;
                a.req_tgt[out] = result;
                if (result < 0)
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.failed), 1ull);
                if (a.diag_lns) {
                    a.diag_lns[out] = lns0;
                    a.diag_evals[out] = evals;
                    a.diag_restarts[out] = draws > 0 ? draws - 1 : 0;
                }
            }
        }
        if constexpr (kCount) { // this task's counts: one atomic per warp
            int64_t ts = task_steps;
            for (int off = 16; off; off >>= 1) {
                task_evals += __shfl_xor_sync(0xffffffffu, task_evals, off);
                ts += __shfl_xor_sync(0xffffffffu, ts, off);
            }
            if (lane == 0 && task_evals)
                atomicAdd(reinterpret_cast<unsigned long long *>(a.evals_total),
                          (unsigned long long)task_evals);
            if (lane == 0 && ts)
                atomicAdd(reinterpret_cast<unsigned long long *>(a.steps_total),
                          (unsigned long long)ts);
        }
    }
}

// ---------------------------------------------------------------------------
// Split kernel: one warp per source, for updates with few sources (the union
// kernel would leave most of the GPU idle while each lane walks a whole frontier
// alone, one dependent node load after another).
//
// The source's frontier walk is shared out among the 32 lanes as contiguous
// ranges of the pre-order node array. A walk over a range [b, e) is the plain
// stackless walk started at b: b is always a node the source's walk visits (the
// root's first child, or the escape of a node the walk descended into), so the
// range holds exactly the source's candidates between b and e, in order. Lane 0
// starts with [root + 1, root end); whenever a lane descends into a rejected node
// p while other lanes are idle, it keeps [b, escape(p)) and hands the rest,
// [escape(p), e), to an idle lane. Ranges therefore stay contiguous and are
// linked in pre-order (each keeps the index of the range that follows it), and
// work is rebalanced at every step instead of by a fixed partition.
//
// Each range's candidates are summed from zero in FP32 with Kahan compensation;
// the ranges' partial sums then form an FP64 inclusive prefix in pre-order (S is
// its total), and each lane draws one of the source's searches: the range holding
// u * S by binary search, inside it by repeating its walk and partial sum, then
// restarts as in the union kernel. The candidates and their order are the union
// kernel's; only the association of the FP32/FP64 sums differs, so a draw can
// differ from the union kernel's only within rounding of a cumulative boundary.
// Ranges per source (the list stops growing there), chosen per launch from theta
// (split_capacity): the frontier, and with it the number of ranges a walk hands out,
// grows about as theta^-2. Too few ranges leave lanes idle once the list is full;
// more cost shared memory, i.e. L1 (the SM's 256 KB hold both) and resident blocks.
// The split updates of the clustered benchmark (updates 4 and 5), per capacity:
// theta 0.3: 320 ranges 1.66 ms, 448 1.22 / 0.43 ms, 512 1.50 / 0.52 ms (53 KB per
// block leave about 28 KB of L1, 448 ranges about 60 KB); theta 0.2: 448 7.11 ms,
// 512 5.62, 640 4.20, 768 3.64 ms; theta 0.5: 320 0.56 ms, 448 0.62 ms.
constexpr int kSplitMinCap = 320, kSplitMaxCap = 1024;
constexpr int kSplitMinRest = 32; // a rest of fewer nodes is not handed out

// The source's candidates in [b, e), compensated sum from zero, until the running
// total exceeds rel: that candidate, else the last with weight, else -1. The same
// arithmetic as bh_split_kernel's range walks, step for step.
__device__ __forceinline__ int32_t range_find(const Node *__restrict__ nodes, int32_t b,
                                              int32_t e, float3 x, int32_t self_node,
                                              uint32_t thr0, float k2, float k2sh, float rel)
{
    int32_t p = b, pick = -1;
    float cum = 0.0f, comp = 0.0f;
    while (p < e) {
        float4 g;
        int2 t;
        load_node(&nodes[p], g, t);
        const float d2 = dist2(x, g);
        const bool has = g.w > 0.0f;
        const bool acc = has && (__float_as_uint(d2) + (uint32_t)t.y > thr0);
        if (acc && p != self_node) {
            const float at = attraction(g.w, d2, k2, k2sh);
            kahan_add(cum, comp, at);
            if (at > 0.0f) pick = p;
            if (__fsub_rn(cum, comp) > rel) return p;
        }
        p = (has && !acc) ? p + 1 : max(t.x, p + 1);
    }
    return pick;
}

__device__ __forceinline__ int warp_sum_i(int v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per warp: the ranges of the current source and their order, in dynamic shared
// memory (cap ranges). The FP64 prefix of the partial sums in pre-order is kept as 32
// block starts: lane k sums the ranges ord[k * per .. (k + 1) * per) on top of
// start[k] (see split_walk).
struct SplitLists {
    double *start;                          // [32] prefix before each lane's block
    int32_t *give_b, *give_e, *give_next;   // [32] hand-over slots of one step
    int32_t *b;                             // [cap] first node of each range
    float *part;                            // [cap] its compensated partial sum
    int16_t *next;                          // [cap] the range after it in pre-order
    int16_t *ord;                           // [cap] ranges in pre-order
    int cap;
};
__host__ __device__ constexpr size_t split_warp_bytes(int cap)
{
    return 32 * sizeof(double) + 3 * 32 * sizeof(int32_t) + (size_t)cap * 12;
}
__device__ __forceinline__ SplitLists split_lists(unsigned char *raw, int w, int cap)
{
    unsigned char *base = raw + (size_t)w * split_warp_bytes(cap); // 8-byte aligned
    SplitLists L;
    L.start = reinterpret_cast<double *>(base);
    L.give_b = reinterpret_cast<int32_t *>(base + 32 * sizeof(double));
    L.give_e = L.give_b + 32;
    L.give_next = L.give_e + 32;
    L.b = L.give_next + 32;
    L.part = reinterpret_cast<float *>(L.b + cap);
    L.next = reinterpret_cast<int16_t *>(L.part + cap);
    L.ord = L.next + cap;
    L.cap = cap;
    return L;
}

// The inclusive prefix of the ranges in pre-order, as split_walk forms it: the
// first position q whose prefix exceeds tgt (tgt < S), and the prefix before q.
__device__ __forceinline__ int split_locate(const SplitLists &L, int n_rec, double tgt,
                                            double &base)
{
    const int per = (n_rec + 31) >> 5;
    const int nb = (n_rec + per - 1) / per; // non-empty blocks
    int k = 0;
    for (int j = 1; j < nb; ++j)
        if (L.start[j] <= tgt) k = j;
    const int q0 = k * per, q1 = min(q0 + per, n_rec);
    double run = 0.0;
    for (int q = q0; q < q1; ++q) {
        const double before = L.start[k] + run;
        run += (double)L.part[L.ord[q]];
        if (L.start[k] + run > tgt || q == q1 - 1) {
            base = before;
            return q;
        }
    }
    base = L.start[k];
    return q0;
}

// The shared walk of one source's frontier (see above). Every lane of the warp
// calls it. Returns the number of ranges and S (every lane); own (this lane's
// evaluations), dmin2 (nearest candidate this lane met) and steps (walk steps,
// lane 0) accumulate.
__device__ __forceinline__ int split_walk(const SearchArgs &a, SplitLists &L, int32_t root,
                                          int32_t root_end, float3 x, int32_t self_node,
                                          uint32_t thr0, float k2, float k2sh, int32_t &own,
                                          float &dmin2, int64_t &steps, double &S)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    int32_t p = 0, e = 0, rid = -1, rnext = -1;
    float cum = 0.0f, comp = 0.0f;
    bool busy = false;
    if (lane == 0) {
        L.b[0] = root + 1;
        L.part[0] = 0.0f;
        L.next[0] = -1;
        rid = 0;
        p = root + 1;
        e = root_end;
        busy = p < e;
    }
    int n_rec = 1;
    __syncwarp();
    for (;;) {
        bool split = false;
        int32_t rest = 0;
        if (busy) {
            float4 g;
            int2 t;
            load_node(&a.nodes[p], g, t);
            const float d2 = dist2(x, g);
            const bool has = g.w > 0.0f;
            const bool acc = has && (__float_as_uint(d2) + (uint32_t)t.y > thr0);
            own += has ? 1 : 0;
            if (acc && p != self_node) {
                kahan_add(cum, comp, attraction(g.w, d2, k2, k2sh));
                dmin2 = fminf(dmin2, d2);
            }
            if (has && !acc) { // descend; the part after p's subtree may go to another lane
                rest = max(t.x, p + 1);
                split = e - rest >= kSplitMinRest;
                p = p + 1;
            } else {
                p = max(t.x, p + 1);
            }
            if (p >= e) { // range done
                L.part[rid] = __fsub_rn(cum, comp);
                L.next[rid] = (int16_t)rnext;
                busy = false;
                split = false;
            }
        }
        const uint32_t idle = __ballot_sync(0xffffffffu, !busy);
        if (idle == 0xffffffffu) break;
        steps += lane == 0 ? 1 : 0;
        const uint32_t spl = __ballot_sync(0xffffffffu, split);
        const int give = min(min(__popc(idle), __popc(spl)), L.cap - n_rec);
        if (give > 0) { // warp-uniform: the r-th splitting lane gives to the r-th idle lane
            const int rs = __popc(spl & lt), ri = __popc(idle & lt);
            if (split && rs < give) {
                L.give_b[rs] = rest;
                L.give_e[rs] = e;
                L.give_next[rs] = rnext;
                e = rest;
                rnext = n_rec + rs;
            }
            __syncwarp();
            if (!busy && ri < give) {
                rid = n_rec + ri;
                p = L.give_b[ri];
                e = L.give_e[ri];
                rnext = L.give_next[ri];
                L.b[rid] = p;
                cum = 0.0f;
                comp = 0.0f;
                busy = true;
            }
            __syncwarp();
            n_rec += give;
        }
    }
    __syncwarp();
    // pre-order of the ranges: follow the links from the first one
    if (lane == 0) {
        int r = 0;
        for (int pos = 0; pos < n_rec; ++pos) { // the links reach every range once
            L.ord[pos] = (int16_t)(r >= 0 ? r : 0);
            if (r >= 0) r = L.next[r];
        }
    }
    __syncwarp();
    // FP64 inclusive prefix in pre-order: lane k sums its block of ranges from zero
    // (blk); its block starts at the sum of blocks 0 .. k-1 (an exclusive warp scan in
    // five steps: GB300 has little FP64 throughput), and the prefix at position q of
    // the block is start + (the block's running sum)
    const int per = (n_rec + 31) >> 5;
    const int q0 = min(lane * per, n_rec), q1 = min(q0 + per, n_rec);
    double blk = 0.0;
    for (int q = q0; q < q1; ++q) blk += (double)L.part[L.ord[q]];
    double start = __shfl_up_sync(0xffffffffu, blk, 1);
    if (lane == 0) start = 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, start, o);
        if (lane >= o) start += t;
    }
    L.start[lane] = start;
    const int nb = (n_rec + per - 1) / per;
    S = __shfl_sync(0xffffffffu, start + blk, nb - 1);
    __syncwarp();
    return n_rec;
}

template <bool kBatched>
__global__ void __launch_bounds__(256) bh_split_kernel(SearchArgs a)
{
    extern __shared__ __align__(16) unsigned char s_raw[]; // 8 x split_warp_bytes(cap)
    const int32_t A = *a.d_A;
    if (!split_launch(a, A)) return; // bh_search_kernel serves this launch
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    SplitLists L = split_lists(s_raw, w, a.split_cap);
    int64_t my_evals = 0, my_steps = 0;
    int32_t root = 0;
    uint32_t thr0 = 0;
    float k2 = 0.0f;
    if constexpr (!kBatched) {
        thr0 = __ldg(&a.sc->thr0);
        k2 = __ldg(&a.sc->k2);
    }
    for (;;) {
        int32_t idx = 0;
        if (lane == 0) idx = atomicAdd(a.work, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= A) break;
        const int32_t s = a.act_src[idx];
        const float4 xp = a.pos[s];
        const float3 x = make_float3(xp.x, xp.y, xp.z);
        const int32_t self_node = a.leaf_of[s];
        if constexpr (kBatched) {
            const int32_t net = a.net[s];
            root = __ldg(&a.root[net]);
            thr0 = __ldg(&a.sc[net].thr0);
            k2 = __ldg(&a.sc[net].k2);
        }
        const int32_t root_end = __ldg(&a.nodes[root].t.escape);
        float k2sh = 0.0f;
        double S = 0.0;
        int32_t own = 0, n_rec = 0;
        for (int attempt = 0; attempt < 2; ++attempt) {
            float dmin2 = __int_as_float(0x7f800000);
            own = 0;
            n_rec = split_walk(a, L, root, root_end, x, self_node, thr0, k2, k2sh, own, dmin2,
                               my_steps, S);
            if (!(S < (double)kTiny)) break;
            // every term underflowed: redo with the exponents shifted by the nearest d^2
            for (int o = 16; o; o >>= 1)
                dmin2 = fminf(dmin2, __shfl_xor_sync(0xffffffffu, dmin2, o));
            if (!(dmin2 < __int_as_float(0x7f800000))) break;
            k2sh = __fmul_rn(k2, dmin2);
            __syncwarp();
        }
        own = warp_sum_i(own);
        if (lane == 0) my_evals += own;

        // ---- draws: the source's searches, one per lane
        const int32_t i = a.perm[s];
        const int32_t nq = max(a.vac_ax[i], 0);
        const int32_t qbase = a.qoff_o[i];
        // ln S for the diagnostics only (an FP64 log per source otherwise wasted)
        const double lns0 = !a.diag_lns ? 0.0
                            : S > 0.0   ? log(S) - (double)k2sh * 0.6931471805599453
                                        : -__longlong_as_double(0x7ff0000000000000LL);
        for (int32_t e = lane; e < nq; e += 32) {
            int32_t result = -1, evals = own, draws = 0;
            if (S > 0.0) {
                const uint32_t u = philox_x((uint32_t)i, a.step, (uint32_t)e << 8, 0u, a.seed);
                const double tgt = (double)u * 2.3283064365386963e-10 * S;
                double base;
                const int lo = split_locate(L, n_rec, tgt, base); // range holding u * S
                const int32_t rb = L.b[L.ord[lo]];
                const int32_t re = lo + 1 < n_rec ? L.b[L.ord[lo + 1]] : root_end;
                const int32_t k = range_find(a.nodes, rb, re, x, self_node, thr0, k2, k2sh,
                                             (float)(tgt - base));
                result = restart_chain(a, k, x, self_node, thr0, k2, i, e, evals, draws,
                                       my_evals);
            }
            const int32_t out = qbase + e;
            a.req_tgt[out] = result;
            if (result < 0) atomicAdd(reinterpret_cast<unsigned long long *>(a.failed), 1ull);
            if (a.diag_lns) {
                a.diag_lns[out] = lns0;
                a.diag_evals[out] = evals;
                a.diag_restarts[out] = draws > 0 ? draws - 1 : 0;
            }
        }
        __syncwarp(); // the lists are reused by the next source
    }
    for (int off = 16; off; off >>= 1) {
        my_evals += __shfl_xor_sync(0xffffffffu, my_evals, off);
        my_steps += __shfl_xor_sync(0xffffffffu, my_steps, off);
    }
    if (a.count && lane == 0 && my_evals)
        atomicAdd(reinterpret_cast<unsigned long long *>(a.evals_total),
                  (unsigned long long)my_evals);
    if (a.count && lane == 0 && my_steps)
        atomicAdd(reinterpret_cast<unsigned long long *>(a.steps_total),
                  (unsigned long long)my_steps);
}

// Deferred restarts, one thread per queued search, in the order of their drawn
// node (pre-order, so neighbouring threads walk the same subtree and share its
// nodes in L1). The arithmetic is restart_chain's: results equal the inline path.
template <bool kBatched>
__global__ void __launch_bounds__(256) bh_restart_kernel(SearchArgs a, const uint32_t *keys,
                                                         const int32_t *vals)
{
    const int32_t P = *a.rq_count;
    int64_t my_evals = 0;
    uint32_t thr0 = 0;
    float k2 = 0.0f;
    if constexpr (!kBatched) {
        thr0 = __ldg(&a.sc->thr0);
        k2 = __ldg(&a.sc->k2);
    }
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P; j += gridDim.x * blockDim.x) {
        const int32_t slot = vals[j];
        const int32_t k = (int32_t)keys[j];
        const int32_t out = a.rq_out[slot], s = a.rq_src[slot];
        const int32_t i = a.perm[s], e = a.req_elem[out];
        const float4 xp = a.pos[s];
        const float3 x = make_float3(xp.x, xp.y, xp.z);
        if constexpr (kBatched) {
            const int32_t net = a.net[s];
            thr0 = __ldg(&a.sc[net].thr0);
            k2 = __ldg(&a.sc[net].k2);
        }
        int32_t evals = a.diag_evals ? a.diag_evals[out] : 0, draws = 0;
        const int32_t result =
            restart_chain(a, k, x, a.leaf_of[s], thr0, k2, i, e, evals, draws, my_evals);
        a.req_tgt[out] = result;
        if (result < 0) atomicAdd(reinterpret_cast<unsigned long long *>(a.failed), 1ull);
        if (a.diag_lns) {
            a.diag_evals[out] = evals;
            a.diag_restarts[out] = draws > 0 ? draws - 1 : 0;
        }
    }
    for (int off = 16; off; off >>= 1) my_evals += __shfl_xor_sync(0xffffffffu, my_evals, off);
    if (a.count && (threadIdx.x & 31) == 0 && my_evals)
        atomicAdd(reinterpret_cast<unsigned long long *>(a.evals_total),
                  (unsigned long long)my_evals);
}

} // namespace

cudaError_t search_constants(relearn_ctx *c, const relearn_params &p, cudaStream_t st)
{
    search_const_kernel<<<(c->num_nets + 255) / 256, 256, 0, st>>>(
        c->d_geom, c->num_nets, p.sigma, p.theta, p.net_sigma, p.net_theta, c->d_sc,
        c->d_status);
    note_launch();
    return cudaGetLastError();
}

cudaError_t search_prepare(relearn_ctx *c, const relearn_params &p, const int32_t *vac_ax,
                           cudaStream_t st)
{
    const int64_t n = c->n;
    QueryOp op;
    op.vac_ax = vac_ax;
    op.perm = c->d_perm;
    op.n = n;
    op.max_searches = c->max_searches;
    op.qoff_o = c->d_qoff_o;
    op.act_src = c->d_act_src;
    op.req_src = c->d_req_src;
    op.req_elem = c->d_req_elem;
    op.req_tgt = c->d_req_tgt;
    op.d_total = c->d_i64 + I64_SCAN_TOTAL;
    op.d_active = c->d_i64 + I64_ACTIVE;
    op.d_Q = c->d_i32 + I32_Q;
    op.d_A = c->d_i32 + I32_ACTIVE;
    op.d_Qout = c->d_i64 + I64_Q;
    op.d_Qsum = c->d_i64 + I64_Q_TOTAL;
    op.status = c->d_status;
    op.g_all = c->d_geom;
    op.B = c->num_nets;
    op.sigma = p.sigma;
    op.theta = p.theta;
    op.net_sigma = p.net_sigma;
    op.net_theta = p.net_theta;
    op.sc_all = c->d_sc;
    const int64_t tiles = std::max<int64_t>(1, (n + pair_scan::kTile - 1) / pair_scan::kTile);
    if (tiles > c->scan.max_blocks) return cudaErrorInvalidValue;
    pair_scan::scan_pair_kernel<QueryOp><<<(unsigned)tiles, pair_scan::kThreads, 0, st>>>(
        op, n, c->scan.flags, reinterpret_cast<longlong2 *>(c->scan.block_sums), c->d_status,
        c->debug_stall_tile);
    c->debug_stall_tile = -1; // one update only
    note_launch();
    return cudaGetLastError();
}

// The split kernel's ranges per source for theta: 448 at 0.3, scaled as theta^-2,
// multiples of 32 in [kSplitMinCap, kSplitMaxCap] (theta 0: the most). Per-network
// thetas (batched form) use the scalar theta of the parameters as the guide.
static int split_capacity(float theta)
{
    if (!(theta > 0.0f)) return kSplitMaxCap;
    const double r = 448.0 * (0.3 / theta) * (0.3 / theta);
    const long c = 32 * std::lround(r / 32.0);
    return (int)std::min<long>(kSplitMaxCap, std::max<long>(kSplitMinCap, c));
}

cudaError_t search_run(relearn_ctx *c, const relearn_params &p, const int32_t *vac_ax,
                       cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->d_i32 + I32_WORK, 0, sizeof(int32_t), st))) return e;
    if ((e = cudaMemsetAsync(c->d_i64 + I64_FAILED, 0, sizeof(int64_t), st))) return e;
    SearchArgs a;
    a.nodes = c->d_nodes;
    a.pos = c->d_pos;
    a.perm = c->d_perm;
    a.act_src = c->d_act_src;
    a.codes = c->d_codes;
    a.leaf_of = c->d_leaf;
    a.vac_ax = vac_ax;
    a.qoff_o = c->d_qoff_o;
    a.d_A = c->d_i32 + I32_ACTIVE;
    a.sc = c->d_sc;
    a.net = c->num_nets > 1 ? c->d_net : nullptr;
    a.root = c->d_root;
    a.work = c->d_i32 + I32_WORK;
    a.req_tgt = c->d_req_tgt;
    a.failed = c->d_i64 + I64_FAILED;
    a.evals_total = c->d_i64 + I64_EVALS_TOTAL;
    a.steps_total = c->d_i64 + I64_STEPS_TOTAL;
    const bool diag = (p.flags & RELEARN_FLAG_DIAG) != 0;
    a.count = diag || (p.flags & RELEARN_FLAG_COUNT) != 0;
    a.diag_lns = diag ? c->d_diag_lns : nullptr;
    a.diag_evals = diag ? c->d_diag_evals : nullptr;
    a.diag_restarts = diag ? c->d_diag_restarts : nullptr;
    a.seed = p.seed;
    a.step = (uint32_t)p.step;
    a.defer = (p.flags & RELEARN_FLAG_REGROUP) != 0;
    a.req_elem = c->d_req_elem;
    a.rq_key = c->d_rq_key;
    a.rq_val = c->d_rq_val;
    a.rq_out = c->d_rq_out;
    a.rq_src = c->d_rq_src;
    a.rq_count = c->d_i32 + I32_RQ;
    if (a.defer && (e = cudaMemsetAsync(a.rq_count, 0, sizeof(int32_t), st))) return e;
    // search_group: 0 = per-warp choice, 1/8/16/32 = fixed width, 2 = split kernel,
    // 1000 + 100 * d + r = per-warp pieces cut at depth-d cells (tuning; r unused),
    // 3000 + f = per-warp choice, split kernel for at most f * 1024 sources (tuning)
    const uint32_t sg = p.search_group;
    a.forced_group = sg < 1000 ? (int)sg : 0;
    const bool depths = sg >= 1000 && sg < 3000;
    a.spread_depth = depths ? (int)((sg - 1000) / 100) : -1;
    a.n_total = c->n;
    void (*kern)(SearchArgs) = a.net ? (a.count ? bh_search_kernel<true, true>
                                                : bh_search_kernel<true, false>)
                                     : (a.count ? bh_search_kernel<false, true>
                                                : bh_search_kernel<false, false>);
    void (*split)(SearchArgs) = a.net ? bh_split_kernel<true> : bh_split_kernel<false>;
    // resident blocks per SM of both kernels, queried once per context, kernel pair and
    // split capacity
    a.split_cap = split_capacity(p.theta);
    const size_t split_smem = 8 * split_warp_bytes(a.split_cap);
    int *occ = c->search_occ[a.net ? 1 : 0];
    int &occ_split = c->split_occ[a.net ? 1 : 0][a.split_cap / 32];
    if (occ[0] == 0) {
        int per_sm = 0;
        // both counting variants have the same launch bounds
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                 &per_sm, a.net ? bh_search_kernel<true, false> : bh_search_kernel<false, false>,
                 256, 0)))
            return e;
        if ((e = cudaFuncSetAttribute(split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(8 * split_warp_bytes(kSplitMaxCap)))))
            return e;
        occ[0] = per_sm < 1 ? 1 : per_sm;
    }
    if (occ_split == 0) {
        int per_sm_split = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_split, split, 256,
                                                               split_smem)))
            return e;
        occ_split = per_sm_split < 1 ? 1 : per_sm_split;
    }
    const int per_sm = occ[0], per_sm_split = occ_split;
    // the union kernel serves 32 sources per warp; with few sources per resident warp
    // it would leave the GPU mostly idle (kernel choice and widths: see kSplitWaves)
    const int64_t warps = (int64_t)c->num_sms * per_sm * 8;
    auto cap = [](int64_t v) { return (int32_t)std::min<int64_t>(v, 1 << 30); };
    a.split_below = sg >= 3000 ? cap((int64_t)(sg - 3000) * 1024) : cap(warps * kSplitWaves);
    // exactly one of the two kernels does the work (each reads the source count)
    kern<<<c->num_sms * per_sm, 256, 0, st>>>(a);
    note_launch();
    split<<<c->num_sms * per_sm_split, 256, split_smem, st>>>(a);
    note_launch();
    if (a.defer) {
        // regroup the deferred restarts by drawn node, then finish them
        int bits = 1;
        while (bits < 32 && ((int64_t)1 << bits) <= c->max_nodes) ++bits;
        int which = 0;
        if ((e = radix_sort_u32(c->d_rq_key, c->d_rq_key_alt, c->d_rq_val, c->d_rq_val_alt,
                                c->max_searches, a.rq_count, bits, c->sort, st, &which)))
            return e;
        void (*rk)(SearchArgs, const uint32_t *, const int32_t *) =
            a.net ? bh_restart_kernel<true> : bh_restart_kernel<false>;
        int per_sm_rk = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_rk, rk, 256, 0))) return e;
        rk<<<c->num_sms * (per_sm_rk > 0 ? per_sm_rk : 1), 256, 0, st>>>(
            a, which ? c->d_rq_key_alt : c->d_rq_key, which ? c->d_rq_val_alt : c->d_rq_val);
        note_launch();
    }
    return cudaGetLastError();
}

} // namespace rl
