// Acceptance, apply, synapse store, deletion and spike delivery
// (Sec. III-A "Update of synapses" and "Update of electrical activity").
//
// Acceptance groups requests by target with a counting pass (histogram, scan,
// scatter). A target with no more requests than vacant dendritic elements
// accepts them all; an over-requested target accepts a request iff fewer than
// vac_de other requests to it have a smaller (priority, source, element) key,
// which is the same set as sorting by that key and taking the first vac_de.
// Requests are numbered in (source id, element) order, so that key orders exactly
// like the 64-bit (priority << 32 | request number), which the scatter stores in the
// target's bucket: ranking a request reads its bucket once, in order.
//
// The store is the synapse multiset. Updates append their new synapses; the
// canonical order (source, then target) with an out-row pointer array and an
// in-view (rows by target, each ordered by source) is restored only when deletion
// or an export needs it. Spike delivery reads the store in any order: each
// synapse of a spiking source adds its sign to its target with an integer atomic
// (exact, so the order does not matter).
#include "internal.h"

namespace rl {

namespace {

#define GRID_STRIDE(i, n)                                                                         \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n);                     \
         i += (int64_t)gridDim.x * blockDim.x)

int id_bits(int64_t n)
{
    int b = 1;
    while (b < 31 && ((int64_t)1 << b) < n) ++b;
    return b;
}

// ---------------------------------------------------------------- acceptance
__global__ void accept_count_kernel(const int32_t *d_Q, const int32_t *__restrict__ req_src,
                                    const int32_t *__restrict__ req_elem,
                                    const int32_t *__restrict__ req_tgt,
                                    uint32_t *__restrict__ prio, int32_t *__restrict__ tcnt,
                                    uint64_t seed, uint32_t step)
{
    const int64_t Q = *d_Q;
    GRID_STRIDE(r, Q)
    {
        int32_t t = req_tgt[r];
        if (t < 0) continue;
        atomicAdd(&tcnt[t], 1);
        prio[r] = philox_x((uint32_t)req_src[r], step, ((uint32_t)req_elem[r] << 8) | 0xFFu, 1u,
                           seed);
    }
}

__device__ __forceinline__ uint64_t request_key(uint32_t prio, int64_t r)
{
    return ((uint64_t)prio << 32) | (uint64_t)(uint32_t)r;
}

// Each request takes a slot of its target's bucket by counting the target's count
// down (the bucket's order does not matter: the decision ranks keys).
__global__ void accept_scatter_kernel(const int32_t *d_Q, const int32_t *__restrict__ req_tgt,
                                      const uint32_t *__restrict__ prio,
                                      const int32_t *__restrict__ toff,
                                      int32_t *__restrict__ tcnt, uint64_t *__restrict__ bucket)
{
    const int64_t Q = *d_Q;
    GRID_STRIDE(r, Q)
    {
        int32_t t = req_tgt[r];
        if (t < 0) continue;
        bucket[toff[t] + atomicSub(&tcnt[t], 1) - 1] = request_key(prio[r], r);
    }
}

// A target's request count is the difference of neighbouring bucket offsets (one
// read of two adjacent words).
__global__ void accept_decide_kernel(const int32_t *d_Q, const int32_t *__restrict__ req_tgt,
                                     const uint32_t *__restrict__ prio,
                                     const int32_t *__restrict__ toff,
                                     const uint64_t *__restrict__ bucket,
                                     const int32_t *__restrict__ vac_de,
                                     uint8_t *__restrict__ acc, int32_t *__restrict__ flag,
                                     int64_t *declined)
{
    const int64_t Q = *d_Q;
    int64_t dec = 0;
    GRID_STRIDE(r, Q)
    {
        int32_t t = req_tgt[r];
        uint8_t a = 0;
        if (t >= 0) {
            int32_t v = vac_de[t];
            if (v < 0) v = 0;
            const int32_t o = toff[t], rt = toff[t + 1] - o;
            if (rt <= v) {
                a = 1;
            } else if (v > 0) {
                const uint64_t kr = request_key(prio[r], r); // keys are distinct
                const uint64_t *bk = bucket + o;
                int32_t below = 0;
                for (int32_t k = 0; k < rt && below < v; ++k) below += bk[k] < kr ? 1 : 0;
                a = below < v ? 1 : 0;
            }
            dec += a ? 0 : 1;
        }
        acc[r] = a;
        flag[r] = a; // scanned by the apply step into the new synapses' positions
    }
    for (int off = 16; off; off >>= 1) dec += __shfl_xor_sync(0xffffffffu, dec, off);
    if ((threadIdx.x & 31) == 0 && dec)
        atomicAdd(reinterpret_cast<unsigned long long *>(declined), (unsigned long long)dec);
}

// ---------------------------------------------------------------- apply
// New store size check: formed = *d_formed; nothing is applied on overflow. The
// store grows here: the apply kernel writes the new synapses from *d_base (the old
// size) on.
__global__ void apply_check_kernel(const int64_t *d_formed, int32_t *d_nsyn, int32_t *d_new,
                                   int32_t *d_base, int64_t *d_nsyn64, int64_t max_synapses,
                                   int32_t *status, int64_t *d_formed_out)
{
    int64_t f = *d_formed;
    const int32_t base = *d_nsyn;
    const bool failed = *(volatile int32_t *)status != 0; // an earlier kernel reported an error
    *d_base = base;
    if (failed || (int64_t)base + f > max_synapses) {
        if (!failed) set_status(status, RELEARN_ERR_CAPACITY);
        *d_new = -1;
        *d_formed_out = 0;
    } else {
        *d_new = (int32_t)f;
        *d_formed_out = f;
        *d_nsyn = base + (int32_t)f;
    }
    *d_nsyn64 = *d_nsyn;
}

__global__ void apply_kernel(const int32_t *d_Q, const int32_t *d_new, const int32_t *d_base,
                             const int32_t *__restrict__ req_src,
                             const int32_t *__restrict__ req_tgt, const uint8_t *__restrict__ acc,
                             const int32_t *__restrict__ newpos, const uint8_t *__restrict__ type,
                             int32_t *vac_ax, int32_t *vac_de, int32_t *__restrict__ syn_src,
                             int32_t *__restrict__ syn_tgt, int8_t *__restrict__ syn_sign)
{
    if (*d_new < 0) return;
    const int64_t Q = *d_Q;
    const int32_t base = *d_base;
    GRID_STRIDE(r, Q)
    {
        if (!acc[r]) continue;
        const int32_t s = req_src[r], t = req_tgt[r];
        atomicSub(&vac_ax[s], 1);
        atomicSub(&vac_de[t], 1);
        const int32_t k = base + newpos[r];
        syn_src[k] = s;
        syn_tgt[k] = t;
        syn_sign[k] = type[s] ? (int8_t)-1 : (int8_t)1;
    }
}

// ---------------------------------------------------------------- store
__global__ void unpack_keys_kernel(const int32_t *d_nsyn, const uint64_t *__restrict__ key,
                                   const int32_t *__restrict__ val, int bits,
                                   int32_t *__restrict__ src, int32_t *__restrict__ tgt,
                                   int8_t *__restrict__ sign)
{
    const int64_t m = *d_nsyn;
    const uint64_t mask = ((uint64_t)1 << bits) - 1;
    GRID_STRIDE(k, m)
    {
        uint64_t kk = key[k];
        src[k] = (int32_t)(kk >> bits);
        tgt[k] = (int32_t)(kk & mask);
        sign[k] = (int8_t)val[k];
    }
}

__global__ void degree_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ src,
                              const int32_t *__restrict__ tgt, int32_t *__restrict__ out_cnt,
                              int32_t *__restrict__ in_cnt)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(k, m)
    {
        atomicAdd(&out_cnt[src[k]], 1);
        atomicAdd(&in_cnt[tgt[k]], 1);
    }
}

// The canonical order without a global sort: each synapse goes to its source's row
// (any order within the row), then takes its rank in the row by (target, place in
// the row). Rows are short (a neuron's bound elements), so ranking by counting is
// cheaper than sorting the whole store; equal (source, target) records are
// identical (the sign follows the source), so their order does not matter.
__global__ void row_scatter_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ src,
                                   const int32_t *__restrict__ tgt, const int8_t *__restrict__ sign,
                                   const int32_t *__restrict__ out_ptr, int32_t *__restrict__ fill,
                                   int32_t *__restrict__ row_src, int32_t *__restrict__ row_tgt,
                                   int32_t *__restrict__ row_sign)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(k, m)
    {
        const int32_t s = src[k];
        const int32_t r = out_ptr[s] + atomicAdd(&fill[s], 1);
        row_src[r] = s;
        row_tgt[r] = tgt[k];
        row_sign[r] = sign[k];
    }
}

__global__ void row_rank_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ row_src,
                                const int32_t *__restrict__ row_tgt,
                                const int32_t *__restrict__ row_sign,
                                const int32_t *__restrict__ out_ptr, int32_t *__restrict__ src,
                                int32_t *__restrict__ tgt, int8_t *__restrict__ sign)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(r, m)
    {
        const int32_t s = row_src[r], t = row_tgt[r];
        const int32_t b = out_ptr[s], e = out_ptr[s + 1];
        int32_t rank = 0;
        for (int32_t j = b; j < e; ++j) {
            const int32_t tj = row_tgt[j];
            rank += (tj < t || (tj == t && j < r)) ? 1 : 0;
        }
        const int32_t w = b + rank;
        src[w] = s;
        tgt[w] = t;
        sign[w] = (int8_t)row_sign[r];
    }
}

// In-view: synapse numbers k (canonical order) grouped by target, each row ordered by
// k (i.e. by source), by the same scatter-then-rank.
__global__ void in_scatter_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ tgt,
                                  const int32_t *__restrict__ in_ptr, int32_t *__restrict__ fill,
                                  int32_t *__restrict__ row_k)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(k, m)
    {
        const int32_t t = tgt[k];
        row_k[in_ptr[t] + atomicAdd(&fill[t], 1)] = (int32_t)k;
    }
}

__global__ void in_rank_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ tgt,
                               const int32_t *__restrict__ in_ptr,
                               const int32_t *__restrict__ row_k, int32_t *__restrict__ in_syn)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(r, m)
    {
        const int32_t k = row_k[r], t = tgt[k];
        const int32_t b = in_ptr[t], e = in_ptr[t + 1];
        int32_t rank = 0;
        for (int32_t j = b; j < e; ++j) rank += row_k[j] < k ? 1 : 0;
        in_syn[b + rank] = k;
    }
}

// ---------------------------------------------------------------- deletion
__global__ void delete_needs_kernel(int64_t n, const int32_t *__restrict__ retract_ax,
                                    const int32_t *__restrict__ retract_de, int32_t *vac_ax,
                                    int32_t *vac_de, const int32_t *__restrict__ out_ptr,
                                    const int32_t *__restrict__ in_ptr,
                                    int32_t *__restrict__ need_ax, int32_t *__restrict__ need_de)
{
    GRID_STRIDE(i, n)
    {
        int32_t ra = retract_ax[i] > 0 ? retract_ax[i] : 0;
        int32_t va = vac_ax[i];
        int32_t ta = ra < va ? ra : (va > 0 ? va : 0);
        vac_ax[i] = va - ta;
        ra -= ta;
        int32_t deg = out_ptr[i + 1] - out_ptr[i];
        need_ax[i] = ra < deg ? ra : deg;
        int32_t rd = retract_de[i] > 0 ? retract_de[i] : 0;
        int32_t vd = vac_de[i];
        int32_t td = rd < vd ? rd : (vd > 0 ? vd : 0);
        vac_de[i] = vd - td;
        rd -= td;
        int32_t din = in_ptr[i + 1] - in_ptr[i];
        need_de[i] = rd < din ? rd : din;
    }
}

__global__ void delete_prio_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ src,
                                   const int32_t *__restrict__ in_syn,
                                   const int32_t *__restrict__ tgt,
                                   const int32_t *__restrict__ out_ptr,
                                   const int32_t *__restrict__ in_ptr,
                                   uint32_t *__restrict__ prio_ax, uint32_t *__restrict__ prio_de,
                                   uint8_t *__restrict__ sel_ax, uint8_t *__restrict__ sel_de,
                                   uint64_t seed, uint32_t step)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(k, m)
    {
        int32_t i = src[k];
        prio_ax[k] = philox_x((uint32_t)i, step, (uint32_t)(k - out_ptr[i]), 2u, seed);
        int32_t j = tgt[in_syn[k]];
        prio_de[k] = philox_x((uint32_t)j, step, (uint32_t)(k - in_ptr[j]), 3u, seed);
        sel_ax[k] = 0;
        sel_de[k] = 0;
    }
}

// Row i picks its `need` slots with the smallest (priority, slot).
__global__ void delete_select_kernel(int64_t n, const int32_t *__restrict__ ptr,
                                     const int32_t *__restrict__ need,
                                     const uint32_t *__restrict__ prio,
                                     const int32_t *__restrict__ map, uint8_t *__restrict__ sel)
{
    GRID_STRIDE(i, n)
    {
        const int32_t want = need[i];
        if (want <= 0) continue;
        const int32_t b = ptr[i], deg = ptr[i + 1] - b;
        for (int32_t k = 0; k < deg; ++k) {
            const uint32_t pk = prio[b + k];
            int32_t below = 0;
            for (int32_t o = 0; o < deg && below < want; ++o) {
                uint32_t po = prio[b + o];
                if (po < pk || (po == pk && o < k)) ++below;
            }
            if (below < want) sel[map ? map[b + k] : b + k] = 1;
        }
    }
}

__global__ void delete_apply_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ src,
                                    const int32_t *__restrict__ tgt,
                                    const uint8_t *__restrict__ sel_ax,
                                    const uint8_t *__restrict__ sel_de, int32_t *vac_ax,
                                    int32_t *vac_de, int32_t *__restrict__ keep)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(k, m)
    {
        const bool a = sel_ax[k], d = sel_de[k];
        if (a && !d) atomicAdd(&vac_de[tgt[k]], 1);
        if (d && !a) atomicAdd(&vac_ax[src[k]], 1);
        keep[k] = (a || d) ? 0 : 1;
    }
}

__global__ void compact_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ src,
                               const int32_t *__restrict__ tgt, const int8_t *__restrict__ sign,
                               const uint8_t *__restrict__ sel_ax,
                               const uint8_t *__restrict__ sel_de,
                               const int32_t *__restrict__ pos, int bits,
                               uint64_t *__restrict__ key, int32_t *__restrict__ val)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(k, m)
    {
        if (sel_ax[k] || sel_de[k]) continue;
        int32_t w = pos[k];
        key[w] = ((uint64_t)(uint32_t)src[k] << bits) | (uint32_t)tgt[k];
        val[w] = sign[k];
    }
}

__global__ void shrink_store_kernel(int32_t *d_nsyn, const int64_t *d_kept, int64_t *d_broken,
                                    int64_t *d_nsyn64)
{
    int64_t kept = *d_kept;
    *d_broken = (int64_t)*d_nsyn - kept;
    *d_nsyn = (int32_t)kept;
    *d_nsyn64 = kept;
}

// ---------------------------------------------------------------- spikes
// input[t] += sign for every synapse s -> t of a spiking source (input zeroed first).
__global__ void spikes_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ src,
                              const int32_t *__restrict__ tgt, const int8_t *__restrict__ sign,
                              const uint8_t *__restrict__ spiked, int32_t *__restrict__ input)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(k, m)
    {
        if (spiked[src[k]]) atomicAdd(&input[tgt[k]], (int32_t)sign[k]);
    }
}

// Firing-rate delivery (Sec. IV-B): the receiver t decides once per step and per
// source s whether s spiked, spiked iff philox({s, t, step, 4}).x < rate[s] * 2^32
// (an exact FP64 comparison); duplicates of (s, t) share that decision (each
// copy computes the same word).
__global__ void rates_kernel(const int32_t *d_nsyn, const int32_t *__restrict__ src,
                             const int32_t *__restrict__ tgt, const int8_t *__restrict__ sign,
                             const float *__restrict__ rate, uint64_t seed, uint32_t step,
                             int32_t *__restrict__ input)
{
    const int64_t m = *d_nsyn;
    GRID_STRIDE(k, m)
    {
        const int32_t s = src[k], t = tgt[k];
        const uint32_t w = philox_x((uint32_t)s, (uint32_t)t, step, 4u, seed);
        if ((double)w < (double)rate[s] * 4294967296.0) atomicAdd(&input[t], (int32_t)sign[k]);
    }
}

} // namespace

cudaError_t deliver_rates(relearn_ctx *c, const float *rate, uint64_t seed, uint32_t step,
                          int32_t *input, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(input, 0, c->n * sizeof(int32_t), st))) return e;
    rates_kernel<<<grid_for(c->max_synapses, 256, c->num_sms), 256, 0, st>>>(
        c->d_i32 + I32_NSYN, c->d_syn_src, c->d_syn_tgt, c->d_syn_sign, rate, seed, step, input);
    note_launch();
    return cudaGetLastError();
}

cudaError_t accept_requests(relearn_ctx *c, const relearn_params &p, const int32_t *vac_de,
                            cudaStream_t st)
{
    cudaError_t e;
    const int64_t n = c->n;
    const int32_t *dQ = c->d_i32 + I32_Q;
    const unsigned gq = grid_for(c->max_searches, 256, c->num_sms);
    if ((e = cudaMemsetAsync(c->d_tcnt, 0, (n + 1) * sizeof(int32_t), st))) return e;
    if ((e = cudaMemsetAsync(c->d_i64 + I64_DECLINED, 0, sizeof(int64_t), st))) return e;
    accept_count_kernel<<<gq, 256, 0, st>>>(dQ, c->d_req_src, c->d_req_elem, c->d_req_tgt,
                                            c->d_req_prio, c->d_tcnt, p.seed, (uint32_t)p.step);
    note_launch();
    if ((e = scan_exclusive(c->d_tcnt, c->d_toff, n + 1, nullptr, nullptr, c->scan, st))) return e;
    accept_scatter_kernel<<<gq, 256, 0, st>>>(dQ, c->d_req_tgt, c->d_req_prio, c->d_toff,
                                              c->d_tcnt, c->d_bucket);
    note_launch();
    accept_decide_kernel<<<gq, 256, 0, st>>>(dQ, c->d_req_tgt, c->d_req_prio, c->d_toff,
                                             c->d_bucket,
                                             vac_de, c->d_req_acc, c->d_newpos,
                                             c->d_i64 + I64_DECLINED);
    note_launch();
    return cudaGetLastError();
}

// The store in canonical order (source, then target) with its views: out-row
// pointers, in-row pointers and the in-view. Counting pass, two scans, then one
// scatter and one in-row ranking per side (see row_scatter_kernel).
cudaError_t canonicalise_store(relearn_ctx *c, cudaStream_t st)
{
    cudaError_t e;
    const int64_t n = c->n;
    const int32_t *dm = c->d_i32 + I32_NSYN;
    const unsigned gs = grid_for(c->max_synapses, 256, c->num_sms);
    int32_t *out_cnt = c->d_cnt, *in_cnt = c->d_tcnt, *fill = c->d_need_ax;
    int32_t *row_src = c->d_val, *row_sign = c->d_val_alt;
    int32_t *row_tgt = reinterpret_cast<int32_t *>(c->d_key32);
    int32_t *row_k = reinterpret_cast<int32_t *>(c->d_key32_alt);
    if ((e = cudaMemsetAsync(out_cnt, 0, (n + 1) * sizeof(int32_t), st))) return e;
    if ((e = cudaMemsetAsync(in_cnt, 0, (n + 1) * sizeof(int32_t), st))) return e;
    degree_kernel<<<gs, 256, 0, st>>>(dm, c->d_syn_src, c->d_syn_tgt, out_cnt, in_cnt);
    note_launch();
    if ((e = scan_exclusive(out_cnt, c->d_out_ptr, n + 1, nullptr, nullptr, c->scan, st)))
        return e;
    if ((e = scan_exclusive(in_cnt, c->d_in_ptr, n + 1, nullptr, nullptr, c->scan, st))) return e;
    if ((e = cudaMemsetAsync(fill, 0, n * sizeof(int32_t), st))) return e;
    row_scatter_kernel<<<gs, 256, 0, st>>>(dm, c->d_syn_src, c->d_syn_tgt, c->d_syn_sign,
                                           c->d_out_ptr, fill, row_src, row_tgt, row_sign);
    note_launch();
    row_rank_kernel<<<gs, 256, 0, st>>>(dm, row_src, row_tgt, row_sign, c->d_out_ptr,
                                        c->d_syn_src, c->d_syn_tgt, c->d_syn_sign);
    note_launch();
    if ((e = cudaMemsetAsync(fill, 0, n * sizeof(int32_t), st))) return e;
    in_scatter_kernel<<<gs, 256, 0, st>>>(dm, c->d_syn_tgt, c->d_in_ptr, fill, row_k);
    note_launch();
    in_rank_kernel<<<gs, 256, 0, st>>>(dm, c->d_syn_tgt, c->d_in_ptr, row_k, c->d_in_syn);
    note_launch();
    c->canonical = true;
    return cudaGetLastError();
}

cudaError_t apply_requests(relearn_ctx *c, int32_t *vac_ax, int32_t *vac_de, const uint8_t *type,
                           cudaStream_t st)
{
    cudaError_t e;
    const int32_t *dQ = c->d_i32 + I32_Q;
    const unsigned gq = grid_for(c->max_searches, 256, c->num_sms);
    // d_newpos holds the acceptance flags (written by the acceptance step)
    if ((e = scan_exclusive(c->d_newpos, c->d_newpos, c->max_searches, dQ,
                            c->d_i64 + I64_SCAN_TOTAL, c->scan, st)))
        return e;
    apply_check_kernel<<<1, 1, 0, st>>>(c->d_i64 + I64_SCAN_TOTAL, c->d_i32 + I32_NSYN,
                                        c->d_i32 + I32_NEW, c->d_i32 + I32_BASE,
                                        c->d_i64 + I64_NSYN, c->max_synapses, c->d_status,
                                        c->d_i64 + I64_FORMED);
    note_launch();
    apply_kernel<<<gq, 256, 0, st>>>(dQ, c->d_i32 + I32_NEW, c->d_i32 + I32_BASE, c->d_req_src,
                                     c->d_req_tgt, c->d_req_acc, c->d_newpos, type, vac_ax,
                                     vac_de, c->d_syn_src, c->d_syn_tgt, c->d_syn_sign);
    note_launch();
    // new synapses sit unsorted at the end of the store until an operation needs the
    // canonical order (deletion, export); spike delivery reads the store in any order
    c->canonical = false;
    return cudaGetLastError();
}

cudaError_t delete_synapses(relearn_ctx *c, const relearn_params &p, const int32_t *retract_ax,
                            const int32_t *retract_de, int32_t *vac_ax, int32_t *vac_de,
                            cudaStream_t st)
{
    cudaError_t e;
    const int64_t n = c->n;
    const int bits = id_bits(c->max_neurons);
    const int32_t *dm = c->d_i32 + I32_NSYN;
    const unsigned gs = grid_for(c->max_synapses, 256, c->num_sms);
    const unsigned gn = grid_for(n, 256, c->num_sms);
    if (!c->canonical && (e = canonicalise_store(c, st))) return e;
    delete_needs_kernel<<<gn, 256, 0, st>>>(n, retract_ax, retract_de, vac_ax, vac_de,
                                            c->d_out_ptr, c->d_in_ptr, c->d_need_ax,
                                            c->d_need_de);
    note_launch();
    delete_prio_kernel<<<gs, 256, 0, st>>>(dm, c->d_syn_src, c->d_in_syn, c->d_syn_tgt,
                                           c->d_out_ptr, c->d_in_ptr, c->d_prio_ax, c->d_prio_de,
                                           c->d_sel_ax, c->d_sel_de, p.seed, (uint32_t)p.step);
    note_launch();
    delete_select_kernel<<<gn, 256, 0, st>>>(n, c->d_out_ptr, c->d_need_ax, c->d_prio_ax, nullptr,
                                             c->d_sel_ax);
    note_launch();
    delete_select_kernel<<<gn, 256, 0, st>>>(n, c->d_in_ptr, c->d_need_de, c->d_prio_de,
                                             c->d_in_syn, c->d_sel_de);
    note_launch();
    delete_apply_kernel<<<gs, 256, 0, st>>>(dm, c->d_syn_src, c->d_syn_tgt, c->d_sel_ax,
                                            c->d_sel_de, vac_ax, vac_de, c->d_keep);
    note_launch();
    if ((e = scan_exclusive(c->d_keep, c->d_keep, c->max_synapses, dm, c->d_i64 + I64_SCAN_TOTAL,
                            c->scan, st)))
        return e;
    compact_kernel<<<gs, 256, 0, st>>>(dm, c->d_syn_src, c->d_syn_tgt, c->d_syn_sign, c->d_sel_ax,
                                       c->d_sel_de, c->d_keep, bits, c->d_key, c->d_val);
    note_launch();
    shrink_store_kernel<<<1, 1, 0, st>>>(c->d_i32 + I32_NSYN, c->d_i64 + I64_SCAN_TOTAL,
                                         c->d_i64 + I64_BROKEN, c->d_i64 + I64_NSYN);
    note_launch();
    unpack_keys_kernel<<<gs, 256, 0, st>>>(dm, c->d_key, c->d_val, bits, c->d_syn_src,
                                           c->d_syn_tgt, c->d_syn_sign);
    note_launch();
    // the kept synapses are in canonical order; their views are rebuilt when an
    // operation next needs them (the next update appends anyway)
    c->canonical = false;
    return cudaGetLastError();
}

namespace {

// Typed dendrite pools: the axons of one type, and writing them back.
__global__ void select_type_kernel(const int32_t *__restrict__ vac_ax,
                                   const uint8_t *__restrict__ type, int kind, int64_t n,
                                   int32_t *__restrict__ out)
{
    GRID_STRIDE(i, n) out[i] = type[i] == kind ? vac_ax[i] : 0;
}

__global__ void merge_type_kernel(const int32_t *__restrict__ part,
                                  const uint8_t *__restrict__ type, int kind, int64_t n,
                                  int32_t *__restrict__ vac_ax)
{
    GRID_STRIDE(i, n)
    {
        if (type[i] == kind) vac_ax[i] = part[i];
    }
}

} // namespace

cudaError_t select_type(relearn_ctx *c, const int32_t *vac_ax, const uint8_t *type, int kind,
                        int32_t *out, cudaStream_t st)
{
    select_type_kernel<<<grid_for(c->n, 256, c->num_sms), 256, 0, st>>>(vac_ax, type, kind, c->n,
                                                                        out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t merge_type(relearn_ctx *c, const int32_t *part, const uint8_t *type, int kind,
                       int32_t *vac_ax, cudaStream_t st)
{
    merge_type_kernel<<<grid_for(c->n, 256, c->num_sms), 256, 0, st>>>(part, type, kind, c->n,
                                                                       vac_ax);
    note_launch();
    return cudaGetLastError();
}

cudaError_t deliver_spikes(relearn_ctx *c, const uint8_t *spiked, int32_t *input,
                           cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(input, 0, c->n * sizeof(int32_t), st))) return e;
    spikes_kernel<<<grid_for(c->max_synapses, 256, c->num_sms), 256, 0, st>>>(
        c->d_i32 + I32_NSYN, c->d_syn_src, c->d_syn_tgt, c->d_syn_sign, spiked, input);
    note_launch();
    return cudaGetLastError();
}

} // namespace rl
