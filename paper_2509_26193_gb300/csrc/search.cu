// Barnes-Hut partner search (Sec. III-B "Division of work", second paragraph;
// acceptance criterion and theta from Sec. II).
//
// One thread per search (neuron i, element e). Searches are scheduled in
// Morton order of their source, 32 consecutive ones per warp, so the lanes of a
// warp walk nearly the same nodes. The walk over a start node's subtree is
// stackless: nodes are stored in pre-order, so "expand" is p + 1 and "accept"
// or "skip" jumps to the node's escape index. Candidates are therefore met in
// Morton (range-start) order, which is the order of the cumulative draw.
//
// Per draw, pass 1 sums the attractions a = count * 2^(-k2 d^2) (k2 = log2(e) /
// sigma^2) of the accepted candidates; pass 2 repeats the identical arithmetic
// (explicit round-to-nearest intrinsics, no contraction freedom) until the
// running sum exceeds u * S, so the drawn candidate is exactly the one whose
// cumulative interval holds u * S. If every term would underflow, pass 1 is
// redone with the exponents shifted by the nearest candidate's d^2 (an exact
// common factor).
#include "internal.h"

namespace rl {

namespace {

__global__ void search_const_kernel(const Geom *g, float sigma, float theta, SearchConst *sc)
{
    double ext = g->ext;
    double th = (double)theta;
    for (int d = 0; d < 12; ++d) {
        double len = ext / (double)(1u << d);
        sc->thr[d] = th > 0.0 ? (float)((len / th) * (len / th)) : __int_as_float(0x7f800000);
    }
    double s = (double)sigma;
    sc->k2 = (float)(1.4426950408889634 / (s * s));
}

__global__ void query_counts_kernel(const int32_t *__restrict__ vac_ax,
                                    const int32_t *__restrict__ perm, int64_t n,
                                    int32_t *__restrict__ cnt_sorted, int32_t *__restrict__ cnt_id)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= n;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (s == n) {
            cnt_sorted[n] = 0;
            cnt_id[n] = 0;
            continue;
        }
        int32_t a = vac_ax[perm[s]];
        cnt_sorted[s] = a > 0 ? a : 0;
        int32_t b = vac_ax[s];
        cnt_id[s] = b > 0 ? b : 0;
    }
}

// Q = total; beyond capacity the update is void (status CAPACITY, Q = 0).
__global__ void query_check_kernel(const int64_t *d_total, int64_t max_searches, int32_t *d_Q,
                                   int64_t *d_Qout, int64_t *d_Qsum, int32_t *status)
{
    int64_t q = *d_total;
    *d_Qout = q;
    if (q > max_searches) {
        set_status(status, RELEARN_ERR_CAPACITY);
        q = 0;
    }
    *d_Q = (int32_t)q;
    *d_Qsum += q;
}

__global__ void query_fill_kernel(const int32_t *__restrict__ vac_ax,
                                  const int32_t *__restrict__ perm, int64_t n,
                                  const int32_t *__restrict__ qoff_s,
                                  const int32_t *__restrict__ qoff_o, const int32_t *d_Q,
                                  int32_t *__restrict__ qsrc, int32_t *__restrict__ req_src,
                                  int32_t *__restrict__ req_elem, int32_t *__restrict__ req_tgt)
{
    if (*d_Q == 0) return;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = vac_ax[perm[s]];
        int32_t b0 = qoff_s[s];
        for (int32_t e = 0; e < a; ++e) qsrc[b0 + e] = (int32_t)s;
        int32_t c = vac_ax[s];
        int32_t b1 = qoff_o[s];
        for (int32_t e = 0; e < c; ++e) {
            req_src[b1 + e] = (int32_t)s;
            req_elem[b1 + e] = e;
            req_tgt[b1 + e] = -1;
        }
    }
}

struct SearchArgs {
    const Node *__restrict__ nodes;
    const float4 *__restrict__ pos;
    const int32_t *__restrict__ perm;
    const int32_t *__restrict__ qsrc;
    const int32_t *__restrict__ qoff_s;
    const int32_t *__restrict__ qoff_o;
    const int32_t *d_Q;
    const SearchConst *sc;
    int32_t *work;
    int32_t *req_tgt;
    int64_t *failed;
    int64_t *evals_total;
    double *diag_lns;
    int32_t *diag_evals;
    int32_t *diag_restarts;
    uint64_t seed;
    uint32_t step;
};

struct WalkOut {
    float sum;
    float dmin2;
    int32_t pick;
    int32_t evals;
};

// Walk the subtree of `start`, visiting exactly the candidates of its frontier.
// FIND = false: total attraction and nearest d^2. FIND = true: first candidate
// whose running sum exceeds `target` (else the last one with weight).
template <bool FIND>
__device__ __forceinline__ WalkOut walk(const Node *__restrict__ nodes, int32_t start, float3 x,
                                        int32_t self, const float *thr, float k2, float k2sh,
                                        float target)
{
    WalkOut o{0.0f, __int_as_float(0x7f800000), -1, 0};
    int32_t p = start + 1;
    const int32_t end = __ldg(&nodes[start].t.escape);
    float cum = 0.0f;
    while (p < end) {
        const float4 g = __ldg(reinterpret_cast<const float4 *>(&nodes[p].g));
        const int4 t = __ldg(reinterpret_cast<const int4 *>(&nodes[p].t));
        const float dx = __fsub_rn(x.x, g.x), dy = __fsub_rn(x.y, g.y), dz = __fsub_rn(x.z, g.z);
        const float d2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
        const bool has = g.w > 0.0f;
        const bool leaf = (t.y & kLeafBit) != 0;
        const bool acc = has && (leaf || d2 > thr[t.y & 15]);
        const bool take = acc && !(leaf && t.z == self);
        if (!FIND) o.evals += has ? 1 : 0;
        if (take) {
            const float a = __fmul_rn(g.w, ex2_approx(__fmaf_rn(-k2, d2, k2sh)));
            cum = __fadd_rn(cum, a);
            if (FIND) {
                if (a > 0.0f) o.pick = p;
                if (cum > target) return o;
            } else {
                o.dmin2 = fminf(o.dmin2, d2);
            }
        }
        // t.x > p holds for every well-formed node; max() keeps the walk finite regardless
        p = (has && !leaf && !acc) ? p + 1 : max(t.x, p + 1);
    }
    o.sum = cum;
    return o;
}

__global__ void __launch_bounds__(256) bh_search_kernel(SearchArgs a)
{
    __shared__ float s_thr[12];
    __shared__ float s_k2;
    if (threadIdx.x < 12) s_thr[threadIdx.x] = a.sc->thr[threadIdx.x];
    if (threadIdx.x == 0) s_k2 = a.sc->k2;
    __syncthreads();
    const float k2 = s_k2;
    const int32_t Q = *a.d_Q;
    const int lane = threadIdx.x & 31;
    int64_t warp_evals = 0; // node evaluations of this lane's searches
    for (;;) {
        int32_t qb = 0;
        if (lane == 0) qb = atomicAdd(a.work, 32);
        qb = __shfl_sync(0xffffffffu, qb, 0);
        if (qb >= Q) break;
        const int32_t q = qb + lane;
        if (q >= Q) continue;
        const int32_t s = a.qsrc[q];
        const int32_t e = q - a.qoff_s[s];
        const int32_t i = a.perm[s];
        const float4 xp = a.pos[s];
        const float3 x = make_float3(xp.x, xp.y, xp.z);
        int32_t start = 0, sdepth = 0, result = -1, evals = 0, draws = 0;
        double lns0 = -__longlong_as_double(0x7ff0000000000000LL);
        for (int hop = 0; hop < 24; ++hop) {
            float k2sh = 0.0f;
            WalkOut w1 = walk<false>(a.nodes, start, x, s, s_thr, k2, 0.0f, 0.0f);
            evals += w1.evals;
            if (w1.sum < 8.673617e-19f && w1.dmin2 < __int_as_float(0x7f800000)) {
                // 2^-60: redo with an exact common factor so nothing underflows
                k2sh = __fmul_rn(k2, w1.dmin2);
                w1 = walk<false>(a.nodes, start, x, s, s_thr, k2, k2sh, 0.0f);
            }
            if (!(w1.sum > 0.0f)) break;
            if (hop == 0)
                lns0 = log((double)w1.sum) - (double)k2sh * 0.6931471805599453;
            const uint32_t u = philox_x((uint32_t)i, a.step, ((uint32_t)e << 8) | (uint32_t)sdepth,
                                        0u, a.seed);
            const float target = (float)((double)u * 2.3283064365386963e-10 * (double)w1.sum);
            WalkOut w2 = walk<true>(a.nodes, start, x, s, s_thr, k2, k2sh, target);
            ++draws;
            const int32_t k = w2.pick;
            const int4 tk = __ldg(reinterpret_cast<const int4 *>(&a.nodes[k].t));
            if (tk.y & kLeafBit) {
                result = a.perm[tk.z];
                break;
            }
            start = k;
            sdepth = tk.y & 15;
        }
        const int32_t slot = a.qoff_o[i] + e;
        warp_evals += evals;
        a.req_tgt[slot] = result;
        if (result < 0) atomicAdd(reinterpret_cast<unsigned long long *>(a.failed), 1ull);
        if (a.diag_lns) {
            a.diag_lns[slot] = lns0;
            a.diag_evals[slot] = evals;
            a.diag_restarts[slot] = draws > 0 ? draws - 1 : 0;
        }
    }
    for (int off = 16; off; off >>= 1) warp_evals += __shfl_xor_sync(0xffffffffu, warp_evals, off);
    if (lane == 0 && warp_evals)
        atomicAdd(reinterpret_cast<unsigned long long *>(a.evals_total),
                  (unsigned long long)warp_evals);
}

inline unsigned grid_for(int64_t n, int threads, int num_sms)
{
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 32;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

} // namespace

cudaError_t search_prepare(relearn_ctx *c, const relearn_params &p, const int32_t *vac_ax,
                           cudaStream_t st)
{
    cudaError_t e;
    const int64_t n = c->n;
    search_const_kernel<<<1, 1, 0, st>>>(c->d_geom, p.sigma, p.theta, c->d_sc);
    note_launch();
    int32_t *cnt_s = c->d_cnt, *cnt_o = c->d_tcnt; // scratch
    query_counts_kernel<<<grid_for(n + 1, 256, c->num_sms), 256, 0, st>>>(vac_ax, c->d_perm, n,
                                                                          cnt_s, cnt_o);
    note_launch();
    if ((e = scan_exclusive(cnt_s, c->d_qoff_s, n + 1, nullptr, c->d_i64 + I64_SCAN_TOTAL,
                            c->scan, st)))
        return e;
    if ((e = scan_exclusive(cnt_o, c->d_qoff_o, n + 1, nullptr, nullptr, c->scan, st))) return e;
    query_check_kernel<<<1, 1, 0, st>>>(c->d_i64 + I64_SCAN_TOTAL, c->max_searches,
                                        c->d_i32 + I32_Q, c->d_i64 + I64_Q,
                                        c->d_i64 + I64_Q_TOTAL, c->d_status);
    note_launch();
    query_fill_kernel<<<grid_for(n, 256, c->num_sms), 256, 0, st>>>(
        vac_ax, c->d_perm, n, c->d_qoff_s, c->d_qoff_o, c->d_i32 + I32_Q, c->d_qsrc,
        c->d_req_src, c->d_req_elem, c->d_req_tgt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t search_run(relearn_ctx *c, const relearn_params &p, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->d_i32 + I32_WORK, 0, sizeof(int32_t), st))) return e;
    if ((e = cudaMemsetAsync(c->d_i64 + I64_FAILED, 0, sizeof(int64_t), st))) return e;
    SearchArgs a;
    a.nodes = c->d_nodes;
    a.pos = c->d_pos;
    a.perm = c->d_perm;
    a.qsrc = c->d_qsrc;
    a.qoff_s = c->d_qoff_s;
    a.qoff_o = c->d_qoff_o;
    a.d_Q = c->d_i32 + I32_Q;
    a.sc = c->d_sc;
    a.work = c->d_i32 + I32_WORK;
    a.req_tgt = c->d_req_tgt;
    a.failed = c->d_i64 + I64_FAILED;
    a.evals_total = c->d_i64 + I64_EVALS_TOTAL;
    const bool diag = (p.flags & RELEARN_FLAG_DIAG) != 0;
    a.diag_lns = diag ? c->d_diag_lns : nullptr;
    a.diag_evals = diag ? c->d_diag_evals : nullptr;
    a.diag_restarts = diag ? c->d_diag_restarts : nullptr;
    a.seed = p.seed;
    a.step = (uint32_t)p.step;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bh_search_kernel, 256, 0)))
        return e;
    if (per_sm < 1) per_sm = 1;
    bh_search_kernel<<<c->num_sms * per_sm, 256, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

} // namespace rl
