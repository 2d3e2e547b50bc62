// C ABI of librelearn (declared in include/relearn.h): argument checks,
// context allocation, and the order of the kernels of each call.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace rl;

namespace {
std::atomic<int64_t> g_launches{0};
} // namespace

void rl::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

relearn_status fail(relearn_ctx *c, relearn_status s, const char *what)
{
    if (c) {
        c->host_error = s;
        snprintf(c->msg, sizeof(c->msg), "%s", what);
    }
    return s;
}

relearn_status cuda_fail(relearn_ctx *c, cudaError_t e, const char *where)
{
    if (c) {
        c->host_error = RELEARN_ERR_CUDA;
        snprintf(c->msg, sizeof(c->msg), "%s: %s", where, cudaGetErrorString(e));
    }
    return RELEARN_ERR_CUDA;
}

#define CK(call, where)                                                                           \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where);                                    \
    } while (0)

template <typename T>
cudaError_t alloc(T **p, int64_t count, std::vector<void *> &owned)
{
    size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) owned.push_back((void *)*p);
    return e;
}

void free_all(relearn_ctx *c)
{
    void **ptrs[] = {
        (void **)&c->d_status,   (void **)&c->d_i64,        (void **)&c->d_i32,
        (void **)&c->d_geom,     (void **)&c->d_sc,         (void **)&c->d_codes,
        (void **)&c->d_off,      (void **)&c->d_ord,        (void **)&c->d_root,
        (void **)&c->d_net,      (void **)&c->d_nkey,       (void **)&c->d_nkey_alt,
        (void **)&c->d_lstate,   (void **)&c->d_lsum,
        (void **)&c->d_rq_key,   (void **)&c->d_rq_key_alt, (void **)&c->d_rq_val,
        (void **)&c->d_rq_val_alt, (void **)&c->d_rq_out,   (void **)&c->d_rq_src,
        (void **)&c->d_codes_alt, (void **)&c->d_perm,      (void **)&c->d_perm_alt,
        (void **)&c->d_pos,      (void **)&c->d_posq,       (void **)&c->d_mask,       (void **)&c->d_base,
        (void **)&c->d_nodes,    (void **)&c->d_parent,     (void **)&c->d_nsize,
        (void **)&c->d_leaf,     (void **)&c->d_acc,
        (void **)&c->d_cnt,      (void **)&c->d_act_off,    (void **)&c->d_qoff_o,
        (void **)&c->d_act_src,  (void **)&c->d_req_src,    (void **)&c->d_req_elem,
        (void **)&c->d_req_tgt,  (void **)&c->d_req_acc,    (void **)&c->d_req_prio,
        (void **)&c->d_bucket,   (void **)&c->d_tcnt,       (void **)&c->d_toff,
        (void **)&c->d_newpos,   (void **)&c->d_diag_lns,
        (void **)&c->d_diag_evals, (void **)&c->d_diag_restarts, (void **)&c->d_syn_src,
        (void **)&c->d_syn_tgt,  (void **)&c->d_syn_sign,   (void **)&c->d_key,
        (void **)&c->d_key_alt,  (void **)&c->d_val,        (void **)&c->d_val_alt,
        (void **)&c->d_key32,    (void **)&c->d_key32_alt,  (void **)&c->d_out_ptr,
        (void **)&c->d_in_ptr,   (void **)&c->d_in_syn,
        (void **)&c->d_prio_ax,  (void **)&c->d_prio_de,
        (void **)&c->d_sel_ax,   (void **)&c->d_sel_de,     (void **)&c->d_need_ax,
        (void **)&c->d_need_de,  (void **)&c->d_keep,       (void **)&c->scan.block_sums,
        (void **)&c->scan.flags, (void **)&c->sort.hist};
    for (void **p : ptrs) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    c->sort.scan.block_sums = nullptr;
    c->sort.scan.flags = nullptr;
    if (c->h_off) cudaFreeHost(c->h_off);
    c->h_off = nullptr;
    if (c->off_ev) cudaEventDestroy(c->off_ev);
    c->off_ev = nullptr;
    for (cudaEvent_t &ev : c->ev)
        if (ev) {
            cudaEventDestroy(ev);
            ev = nullptr;
        }
    for (auto &pair : c->kev)
        for (cudaEvent_t &ev : pair)
            if (ev) {
                cudaEventDestroy(ev);
                ev = nullptr;
            }
}

bool params_ok(const relearn_params *p)
{
    return p && (p->net_sigma || (p->sigma > 0.0f && p->sigma < 3.0e38f)) &&
           (p->net_theta || (p->theta >= 0.0f && p->theta < 3.0e38f)) &&
           p->step <= 0xffffffffull &&
           (p->search_group == 0 || p->search_group == 1 || p->search_group == 2 ||
            p->search_group == 8 || p->search_group == 16 || p->search_group == 32 ||
            (p->search_group >= 1000 && p->search_group <= 2010 &&
             (p->search_group - 1000) % 100 <= 10) ||
            (p->search_group >= 3000 && p->search_group <= 3999));
}

relearn_status read_status(relearn_ctx *c)
{
    int32_t st = 0;
    cudaError_t e = cudaMemcpy(&st, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading device status");
    if (st != 0) {
        cudaMemset(c->d_status, 0, sizeof(int32_t));
        return fail(c, (relearn_status)st,
                    st == RELEARN_ERR_CAPACITY  ? "capacity exceeded on the device (searches or "
                                                  "synapses); nothing was applied"
                    : st == RELEARN_ERR_TIMEOUT ? "a bounded wait of the bottom-up update gave "
                                                  "up; nothing was applied"
                                                : "device-side error; nothing was applied");
    }
    return RELEARN_OK;
}

relearn_status sync(relearn_ctx *c)
{
    cudaError_t e = cudaStreamSynchronize(c->last_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    return read_status(c);
}

} // namespace

extern "C" {

relearn_status relearn_create(relearn_ctx **out, int device, int64_t max_neurons,
                              int64_t max_synapses, int64_t max_searches)
{
    return relearn_create_batched(out, device, max_neurons, max_synapses, max_searches, 1);
}

relearn_status relearn_create_batched(relearn_ctx **out, int device, int64_t max_neurons,
                                      int64_t max_synapses, int64_t max_searches,
                                      int32_t max_networks)
{
    if (!out) return RELEARN_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_neurons < 1 || max_neurons > (int64_t)0x3fffffff || max_synapses < 1 ||
        max_synapses > (int64_t)0x7ffffff0 || max_searches < 0 ||
        max_searches > (int64_t)0x7ffffff0 || max_networks < 1 ||
        max_networks > RELEARN_MAX_NETWORKS || max_networks > max_neurons)
        return RELEARN_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return RELEARN_ERR_INVALID_ARG;
    DeviceGuard g(device);
    if (!g.ok) return RELEARN_ERR_CUDA;
    relearn_ctx *c = new (std::nothrow) relearn_ctx();
    if (!c) return RELEARN_ERR_OOM;
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (c->num_sms < 1) c->num_sms = 1;
    c->max_neurons = max_neurons;
    c->max_nets = max_networks;
    c->max_synapses = max_synapses;
    c->max_searches = max_searches ? max_searches : std::min<int64_t>(8 * max_neurons, 0x7ffffff0);
    c->max_nodes = 2 * max_neurons + 1;
    const int64_t N = max_neurons, S = max_synapses, QC = c->max_searches, M = c->max_nodes;
    std::vector<void *> owned;
    cudaError_t e = cudaSuccess;
#define A(ptr, cnt)                                                                               \
    if (e == cudaSuccess) e = alloc(&c->ptr, (cnt), owned)
    A(d_status, 1);
    A(d_i64, 16);
    A(d_i32, 32);
    const int64_t NB = max_networks;
    A(d_geom, NB);
    A(d_sc, NB);
    A(d_off, NB + 1);
    A(d_ord, 6 * NB);
    A(d_root, NB);
    A(d_lstate, N);
    A(d_lsum, 4);
    if (NB > 1) {
        A(d_net, N);
        A(d_nkey, N);
        A(d_nkey_alt, N);
    }
    A(d_codes, N);
    A(d_codes_alt, N);
    A(d_perm, N);
    A(d_perm_alt, N);
    A(d_pos, N);
    A(d_posq, N);
    A(d_mask, N);
    A(d_base, N + 1);
    A(d_nodes, M + 4); // + sentinels past the last node
    A(d_parent, M);
    A(d_nsize, M);
    A(d_leaf, N);
    A(d_acc, 4 * M + 8 * (N / 1024 + 2)); // L4 prefix (n + 1) and the prefix tiles' sums
    A(d_cnt, N + 1);
    A(d_act_off, N + 1);
    A(d_qoff_o, N + 1);
    A(d_act_src, N);
    A(d_req_src, QC);
    A(d_req_elem, QC);
    A(d_req_tgt, QC);
    A(d_req_acc, QC);
    A(d_req_prio, QC);
    A(d_bucket, QC);
    A(d_tcnt, N + 1);
    A(d_toff, N + 1);
    A(d_newpos, QC + 1);
    A(d_rq_key, QC);
    A(d_rq_key_alt, QC);
    A(d_rq_val, QC);
    A(d_rq_val_alt, QC);
    A(d_rq_out, QC);
    A(d_rq_src, QC);
    A(d_diag_lns, QC);
    A(d_diag_evals, QC);
    A(d_diag_restarts, QC);
    A(d_syn_src, S);
    A(d_syn_tgt, S);
    A(d_syn_sign, S);
    A(d_key, S);
    A(d_key_alt, S);
    A(d_val, std::max(S, N));
    A(d_val_alt, std::max(S, N));
    A(d_key32, S);
    A(d_key32_alt, S);
    A(d_out_ptr, N + 1);
    A(d_in_ptr, N + 1);
    A(d_in_syn, S);
    A(d_prio_ax, S);
    A(d_prio_de, S);
    A(d_sel_ax, S);
    A(d_sel_de, S);
    A(d_need_ax, N);
    A(d_need_de, N);
    A(d_keep, S + 1);
    const int64_t sort_blocks = sort_blocks_needed(std::max({N, S, QC}));
    A(sort.hist, 256 * sort_blocks);
    int64_t scan_blocks = std::max({scan_blocks_needed(N + 1), scan_blocks_needed(QC),
                                    scan_blocks_needed(S), scan_blocks_needed(256 * sort_blocks)});
    A(scan.block_sums, 4 * scan_blocks); // a pair scan keeps two sums per tile
    A(scan.flags, scan_blocks + 3);
#undef A
    if (e == cudaSuccess) {
        c->scan.max_blocks = scan_blocks;
        c->scan.status = c->d_status;
        c->scan.grid_cap = scan_grid_cap(c->num_sms);
        c->sort.max_blocks = sort_blocks;
        c->sort.scan = c->scan;
        for (cudaEvent_t &ev : c->ev)
            if (e == cudaSuccess) e = cudaEventCreate(&ev);
        for (auto &pair : c->kev)
            for (cudaEvent_t &ev : pair)
                if (e == cudaSuccess) e = cudaEventCreate(&ev);
    }
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_off, (NB + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->off_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemset(c->scan.flags, 0, (c->scan.max_blocks + 3) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_i64, 0, 16 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_i32, 0, 32 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        relearn_status s = (e == cudaErrorMemoryAllocation) ? RELEARN_ERR_OOM : RELEARN_ERR_CUDA;
        cudaGetLastError();
        free_all(c);
        delete c;
        return s;
    }
    *out = c;
    return RELEARN_OK;
}

relearn_status relearn_destroy(relearn_ctx *c)
{
    if (!c) return RELEARN_OK;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
    return RELEARN_OK;
}

relearn_status relearn_build_octree(relearn_ctx *c, int64_t n, const float *x, const float *y,
                                    const float *z, const int32_t *vac_de, const float *box_lo3,
                                    const float *box_hi3, void *stream)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (n < 1 || n > c->max_neurons)
        return fail(c, RELEARN_ERR_INVALID_ARG, "build_octree: n out of range");
    if (!x || !y || !z) return fail(c, RELEARN_ERR_INVALID_ARG, "build_octree: NULL position");
    if ((box_lo3 == nullptr) != (box_hi3 == nullptr))
        return fail(c, RELEARN_ERR_INVALID_ARG, "build_octree: give both box corners or none");
    if (box_lo3)
        for (int a = 0; a < 3; ++a)
            if (!(box_hi3[a] >= box_lo3[a]))
                return fail(c, RELEARN_ERR_INVALID_ARG, "build_octree: box_hi < box_lo");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, RELEARN_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    const bool reset_store = !c->built || n != c->n;
    c->n = n;
    c->num_nets = 1;
    CK(octree_build(c, n, 1, x, y, z, box_lo3, box_hi3, st), "octree build");
    if (vac_de) CK(octree_reduce(c, vac_de, st), "octree reduce");
    if (reset_store) {
        CK(cudaMemsetAsync(c->d_i32 + I32_NSYN, 0, sizeof(int32_t), st), "store reset");
        CK(cudaMemsetAsync(c->d_i64 + I64_NSYN, 0, sizeof(int64_t), st), "store reset");
        c->canonical = false; // an empty store; its views are formed when first needed
    }
    c->built = true;
    c->diag_valid = false;
    c->length_valid = false;
    return RELEARN_OK;
}

relearn_status relearn_build_octree_batch(relearn_ctx *c, int32_t num_networks,
                                          const int64_t *offsets, const float *x, const float *y,
                                          const float *z, const int32_t *vac_de, void *stream)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (num_networks < 1 || num_networks > c->max_nets)
        return fail(c, RELEARN_ERR_INVALID_ARG, "build_octree_batch: num_networks out of range");
    if (!offsets || !x || !y || !z)
        return fail(c, RELEARN_ERR_INVALID_ARG, "build_octree_batch: NULL argument");
    if (offsets[0] != 0)
        return fail(c, RELEARN_ERR_INVALID_ARG, "build_octree_batch: offsets[0] != 0");
    for (int32_t b = 0; b < num_networks; ++b)
        if (!(offsets[b + 1] > offsets[b]))
            return fail(c, RELEARN_ERR_INVALID_ARG,
                        "build_octree_batch: offsets not strictly increasing");
    const int64_t n = offsets[num_networks];
    if (n > c->max_neurons)
        return fail(c, RELEARN_ERR_INVALID_ARG, "build_octree_batch: n > max_neurons");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, RELEARN_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    // The staging buffer may still feed the previous build's copy (not while capturing:
    // then nothing has run yet).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs), "capture status");
    if (cs == cudaStreamCaptureStatusNone) CK(cudaEventSynchronize(c->off_ev), "staging wait");
    memcpy(c->h_off, offsets, (size_t)(num_networks + 1) * sizeof(int64_t));
    CK(cudaMemcpyAsync(c->d_off, c->h_off, (num_networks + 1) * sizeof(int64_t),
                       cudaMemcpyHostToDevice, st),
       "offsets");
    CK(cudaEventRecord(c->off_ev, st), "event");
    const bool reset_store = !c->built || n != c->n;
    c->n = n;
    c->num_nets = num_networks;
    CK(octree_build(c, n, num_networks, x, y, z, nullptr, nullptr, st), "octree build");
    if (vac_de) CK(octree_reduce(c, vac_de, st), "octree reduce");
    if (reset_store) {
        CK(cudaMemsetAsync(c->d_i32 + I32_NSYN, 0, sizeof(int32_t), st), "store reset");
        CK(cudaMemsetAsync(c->d_i64 + I64_NSYN, 0, sizeof(int64_t), st), "store reset");
        c->canonical = false; // an empty store; its views are formed when first needed
    }
    c->built = true;
    c->diag_valid = false;
    c->length_valid = false;
    return RELEARN_OK;
}

// A phase event of a timed update. Under stream capture it is recorded as an
// event-record node of the graph, so every replay records it and the phase times of
// the last replay can be read; otherwise an ordinary record.
static cudaError_t record_phase(cudaEvent_t ev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cudaEventRecordWithFlags(ev, st,
                                    cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                        : cudaEventRecordDefault);
}

relearn_status relearn_update_connectivity(relearn_ctx *c, const relearn_params *p,
                                           int32_t *vac_ax, int32_t *vac_de,
                                           const uint8_t *type, relearn_update_stats *stats,
                                           void *stream)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (!c->built) return fail(c, RELEARN_ERR_STATE, "update before build_octree");
    if (!params_ok(p)) return fail(c, RELEARN_ERR_INVALID_ARG, "update: bad params");
    if (!vac_ax || !vac_de || !type)
        return fail(c, RELEARN_ERR_INVALID_ARG, "update: NULL array");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, RELEARN_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    const bool timed = stats || (p->flags & RELEARN_FLAG_TIMING);
    c->timed = timed;
    c->length_valid = false;
    if (timed) CK(record_phase(c->ev[0], st), "event");
    CK(octree_reduce(c, vac_de, st), "reduce");
    if (timed) CK(record_phase(c->ev[1], st), "event");
    CK(search_prepare(c, *p, vac_ax, st), "search prepare");
    if (timed) CK(record_phase(c->ev[2], st), "event");
    const bool ring = (p->flags & RELEARN_FLAG_TIMING) && c->nkev < 64;
    if (ring) CK(record_phase(c->kev[c->nkev][0], st), "event");
    CK(search_run(c, *p, vac_ax, st), "search");
    if (ring) CK(record_phase(c->kev[c->nkev++][1], st), "event");
    if (timed) CK(record_phase(c->ev[3], st), "event");
    CK(accept_requests(c, *p, vac_de, st), "accept");
    if (timed) CK(record_phase(c->ev[4], st), "event");
    CK(apply_requests(c, vac_ax, vac_de, type, st), "apply");
    if (timed) CK(record_phase(c->ev[5], st), "event");
    c->diag_valid = (p->flags & RELEARN_FLAG_DIAG) != 0;
    c->stats_valid = true;
    if (stats) return relearn_get_last_stats(c, stats);
    return RELEARN_OK;
}

relearn_status relearn_update_connectivity_typed(relearn_ctx *c, const relearn_params *p,
                                                 int32_t *vac_ax, int32_t *vac_de_exc,
                                                 int32_t *vac_de_inh, const uint8_t *type,
                                                 relearn_update_stats *stats, void *stream)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (!c->built) return fail(c, RELEARN_ERR_STATE, "update before build_octree");
    if (!params_ok(p)) return fail(c, RELEARN_ERR_INVALID_ARG, "update_typed: bad params");
    if (!vac_ax || !vac_de_exc || !vac_de_inh || !type)
        return fail(c, RELEARN_ERR_INVALID_ARG, "update_typed: NULL array");
    if (vac_de_exc == vac_de_inh)
        return fail(c, RELEARN_ERR_INVALID_ARG, "update_typed: the two pools must differ");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, RELEARN_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *part = c->d_need_ax; // scratch [n]: free outside deletion
    relearn_update_stats sum{};
    for (int kind = 0; kind < 2; ++kind) {
        CK(select_type(c, vac_ax, type, kind, part, st), "select type");
        relearn_update_stats one{};
        relearn_status s = relearn_update_connectivity(c, p, part, kind ? vac_de_inh : vac_de_exc,
                                                       type, stats ? &one : nullptr, stream);
        if (s != RELEARN_OK) return s;
        CK(merge_type(c, part, type, kind, vac_ax, st), "merge type");
        if (stats) {
            sum.searches += one.searches;
            sum.failed += one.failed;
            sum.requests_declined += one.requests_declined;
            sum.formed += one.formed;
            sum.synapses = one.synapses;
            sum.ms_reduce += one.ms_reduce;
            sum.ms_search += one.ms_search;
            sum.ms_search_kernel += one.ms_search_kernel;
            sum.ms_accept += one.ms_accept;
            sum.ms_apply += one.ms_apply;
            sum.ms_total += one.ms_total;
            sum.searches_total = one.searches_total;
            sum.evals_total = one.evals_total;
            sum.walk_steps_total = one.walk_steps_total;
            sum.length_evals_total = one.length_evals_total;
        }
    }
    if (stats) *stats = sum;
    return RELEARN_OK;
}

relearn_status relearn_debug_stall_scan(relearn_ctx *c, int64_t tile)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    c->debug_stall_tile = tile < 0 ? -1 : tile;
    return RELEARN_OK;
}

relearn_status relearn_mean_length(relearn_ctx *c, const relearn_params *p,
                                   const int32_t *vac_ax, const int32_t *vac_de, float *ell,
                                   double *mean, void *stream)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (!c->built) return fail(c, RELEARN_ERR_STATE, "mean_length before build_octree");
    if (c->num_nets != 1)
        return fail(c, RELEARN_ERR_STATE, "mean_length: needs a single-network build");
    if (!params_ok(p)) return fail(c, RELEARN_ERR_INVALID_ARG, "mean_length: bad params");
    if (!vac_ax || !vac_de || !mean)
        return fail(c, RELEARN_ERR_INVALID_ARG, "mean_length: NULL argument");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, RELEARN_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    c->length_valid = false;
    CK(octree_reduce(c, vac_de, st), "reduce");
    CK(search_constants(c, *p, st), "constants");
    CK(length_forward(c, vac_ax, ell, mean, st), "mean_length");
    c->length_valid = true;
    c->length_ran = true;
    return RELEARN_OK;
}

relearn_status relearn_mean_length_backward(relearn_ctx *c, const int32_t *vac_ax,
                                            const int32_t *vac_de, const double *grad_mean,
                                            float *gx, float *gy, float *gz, double *gsigma,
                                            void *stream)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (!c->length_valid)
        return fail(c, RELEARN_ERR_STATE, "mean_length_backward without its forward");
    if (!vac_ax || !vac_de || !gx || !gy || !gz)
        return fail(c, RELEARN_ERR_INVALID_ARG, "mean_length_backward: NULL argument");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, RELEARN_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    CK(length_backward(c, vac_ax, vac_de, grad_mean, gx, gy, gz, gsigma, st),
       "mean_length_backward");
    return RELEARN_OK;
}

relearn_status relearn_delete_synapses(relearn_ctx *c, const relearn_params *p,
                                       const int32_t *retract_ax, const int32_t *retract_de,
                                       int32_t *vac_ax, int32_t *vac_de, int64_t *broken,
                                       void *stream)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (!c->built) return fail(c, RELEARN_ERR_STATE, "delete before build_octree");
    if (!p || p->step > 0xffffffffull) return fail(c, RELEARN_ERR_INVALID_ARG, "delete: params");
    if (!retract_ax || !retract_de || !vac_ax || !vac_de)
        return fail(c, RELEARN_ERR_INVALID_ARG, "delete: NULL array");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, RELEARN_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    CK(delete_synapses(c, *p, retract_ax, retract_de, vac_ax, vac_de, st), "delete");
    if (broken) {
        relearn_status s = sync(c);
        CK(cudaMemcpy(broken, c->d_i64 + I64_BROKEN, sizeof(int64_t), cudaMemcpyDeviceToHost),
           "copy");
        return s;
    }
    return RELEARN_OK;
}

relearn_status relearn_deliver_spikes(relearn_ctx *c, const uint8_t *spiked, int32_t *input,
                                      void *stream)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (!c->built) return fail(c, RELEARN_ERR_STATE, "deliver_spikes before build_octree");
    if (!spiked || !input) return fail(c, RELEARN_ERR_INVALID_ARG, "deliver_spikes: NULL array");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, RELEARN_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    CK(deliver_spikes(c, spiked, input, st), "deliver spikes");
    return RELEARN_OK;
}

relearn_status relearn_deliver_rates(relearn_ctx *c, const float *rate, uint64_t seed,
                                     uint64_t step, int32_t *input, void *stream)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (!c->built) return fail(c, RELEARN_ERR_STATE, "deliver_rates before build_octree");
    if (!rate || !input) return fail(c, RELEARN_ERR_INVALID_ARG, "deliver_rates: NULL array");
    if (step > 0xffffffffull) return fail(c, RELEARN_ERR_INVALID_ARG, "deliver_rates: step");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, RELEARN_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    CK(deliver_rates(c, rate, seed, (uint32_t)step, input, st), "deliver rates");
    return RELEARN_OK;
}

relearn_status relearn_get_synapses(relearn_ctx *c, int64_t capacity, int64_t *count,
                                    int32_t *src, int32_t *tgt, int8_t *sign)
{
    if (!c || !count) return RELEARN_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (c->built && !c->canonical) CK(canonicalise_store(c, c->last_stream), "canonicalise");
    relearn_status s = sync(c);
    int32_t m = 0;
    CK(cudaMemcpy(&m, c->d_i32 + I32_NSYN, sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
    *count = m;
    if (src || tgt || sign) {
        if (capacity < m) return fail(c, RELEARN_ERR_INVALID_ARG, "get_synapses: capacity");
        if (src) CK(cudaMemcpy(src, c->d_syn_src, m * 4, cudaMemcpyDeviceToHost), "copy");
        if (tgt) CK(cudaMemcpy(tgt, c->d_syn_tgt, m * 4, cudaMemcpyDeviceToHost), "copy");
        if (sign) CK(cudaMemcpy(sign, c->d_syn_sign, m, cudaMemcpyDeviceToHost), "copy");
    }
    return s;
}

relearn_status relearn_set_synapses(relearn_ctx *c, int64_t count, const int32_t *src,
                                    const int32_t *tgt, const int8_t *sign)
{
    if (!c) return RELEARN_ERR_INVALID_ARG;
    if (!c->built) return fail(c, RELEARN_ERR_STATE, "set_synapses before build_octree");
    if (count < 0 || count > c->max_synapses)
        return fail(c, RELEARN_ERR_INVALID_ARG, "set_synapses: count out of range");
    if (count > 0 && (!src || !tgt || !sign))
        return fail(c, RELEARN_ERR_INVALID_ARG, "set_synapses: NULL array");
    for (int64_t k = 0; k < count; ++k)
        if (src[k] < 0 || src[k] >= c->n || tgt[k] < 0 || tgt[k] >= c->n ||
            (sign[k] != 1 && sign[k] != -1))
            return fail(c, RELEARN_ERR_INVALID_ARG, "set_synapses: id or sign out of range");
    DeviceGuard g(c->device);
    relearn_status s0 = sync(c);
    if (s0 != RELEARN_OK) return s0;
    cudaStream_t st = c->last_stream;
    if (count > 0) {
        CK(cudaMemcpy(c->d_syn_src, src, count * 4, cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(c->d_syn_tgt, tgt, count * 4, cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(c->d_syn_sign, sign, count, cudaMemcpyHostToDevice), "copy");
    }
    int32_t m = (int32_t)count;
    int64_t m64 = count;
    CK(cudaMemcpy(c->d_i32 + I32_NSYN, &m, sizeof(m), cudaMemcpyHostToDevice), "copy");
    CK(cudaMemcpy(c->d_i64 + I64_NSYN, &m64, sizeof(m64), cudaMemcpyHostToDevice), "copy");
    CK(canonicalise_store(c, st), "canonicalise");
    return sync(c);
}

relearn_status relearn_get_requests(relearn_ctx *c, int64_t capacity, int64_t *count,
                                    int32_t *tgt, uint8_t *accept)
{
    if (!c || !count) return RELEARN_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    relearn_status s = sync(c);
    int32_t q = 0;
    CK(cudaMemcpy(&q, c->d_i32 + I32_Q, sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
    *count = q;
    if (tgt || accept) {
        if (capacity < q) return fail(c, RELEARN_ERR_INVALID_ARG, "get_requests: capacity");
        if (tgt) CK(cudaMemcpy(tgt, c->d_req_tgt, (size_t)q * 4, cudaMemcpyDeviceToHost), "copy");
        if (accept)
            CK(cudaMemcpy(accept, c->d_req_acc, (size_t)q, cudaMemcpyDeviceToHost), "copy");
    }
    return s;
}

relearn_status relearn_get_search_diag(relearn_ctx *c, int64_t capacity, int64_t *count,
                                       double *ln_s0, int32_t *evals, int32_t *restarts)
{
    if (!c || !count) return RELEARN_ERR_INVALID_ARG;
    if (!c->diag_valid) return fail(c, RELEARN_ERR_STATE, "no update ran with RELEARN_FLAG_DIAG");
    DeviceGuard g(c->device);
    relearn_status s = sync(c);
    int32_t q = 0;
    CK(cudaMemcpy(&q, c->d_i32 + I32_Q, sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
    *count = q;
    if (ln_s0 || evals || restarts) {
        if (capacity < q) return fail(c, RELEARN_ERR_INVALID_ARG, "get_search_diag: capacity");
        if (ln_s0) CK(cudaMemcpy(ln_s0, c->d_diag_lns, (size_t)q * 8, cudaMemcpyDeviceToHost), "copy");
        if (evals) CK(cudaMemcpy(evals, c->d_diag_evals, (size_t)q * 4, cudaMemcpyDeviceToHost), "copy");
        if (restarts)
            CK(cudaMemcpy(restarts, c->d_diag_restarts, (size_t)q * 4, cudaMemcpyDeviceToHost),
               "copy");
    }
    return s;
}

relearn_status relearn_get_tree(relearn_ctx *c, int64_t capacity, int64_t *num_nodes,
                                int32_t *depth, int32_t *first, int32_t *size, int32_t *is_leaf,
                                int32_t *neuron, int32_t *count, float *cx, float *cy, float *cz,
                                int32_t *perm)
{
    if (!c || !num_nodes) return RELEARN_ERR_INVALID_ARG;
    if (!c->built) return fail(c, RELEARN_ERR_STATE, "get_tree before build_octree");
    DeviceGuard g(c->device);
    relearn_status s = sync(c);
    int64_t m = 0;
    CK(cudaMemcpy(&m, c->d_i64 + I64_NODES, sizeof(m), cudaMemcpyDeviceToHost), "copy");
    *num_nodes = m;
    const int64_t n = c->n;
    std::vector<int32_t> hp;
    if (perm || neuron) {
        hp.resize(n);
        CK(cudaMemcpy(hp.data(), c->d_perm, n * 4, cudaMemcpyDeviceToHost), "copy");
        if (perm) memcpy(perm, hp.data(), n * 4);
    }
    if (depth || first || size || is_leaf || neuron || count || cx || cy || cz) {
        if (capacity < m) return fail(c, RELEARN_ERR_INVALID_ARG, "get_tree: capacity");
        std::vector<Node> h(m);
        std::vector<int32_t> par(m);
        CK(cudaMemcpy(h.data(), c->d_nodes, m * sizeof(Node), cudaMemcpyDeviceToHost), "copy");
        CK(cudaMemcpy(par.data(), c->d_parent, m * sizeof(int32_t), cudaMemcpyDeviceToHost),
           "copy");
        for (int64_t v = 0; v < m; ++v) {
            const Node &nd = h[v];
            const bool leaf = node_is_leaf(nd.t.shift);
            const int32_t f = nd.t.neuron;
            const int32_t fe = nd.t.escape < m ? h[nd.t.escape].t.neuron : (int32_t)n;
            // a leaf sits one level below its parent (depth 11 inside a bucket)
            const int dep = leaf ? (par[v] >= 0 ? depth_of(h[par[v]].t.shift) + 1 : 0)
                                 : depth_of(nd.t.shift);
            if (depth) depth[v] = dep;
            if (first) first[v] = f;
            if (size) size[v] = leaf ? 1 : fe - f;
            if (is_leaf) is_leaf[v] = leaf;
            if (neuron) neuron[v] = leaf ? hp[f] : -1;
            if (count) count[v] = nd.t.icount;
            if (cx) cx[v] = nd.g.cx;
            if (cy) cy[v] = nd.g.cy;
            if (cz) cz[v] = nd.g.cz;
        }
    }
    return s;
}

} // extern "C"

namespace {
__global__ void philox_kernel(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint4 r = philox4x32_10(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]),
                                make_uint2(key[2 * i], key[2 * i + 1]));
        out[4 * i] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}
} // namespace

extern "C" {

relearn_status relearn_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                                     int64_t count, void *stream)
{
    if (count < 0 || (count > 0 && (!ctr || !key || !out))) return RELEARN_ERR_INVALID_ARG;
    if (count == 0) return RELEARN_OK;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    philox_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(ctr, key, out, count);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? RELEARN_OK : RELEARN_ERR_CUDA;
}

relearn_status relearn_get_last_stats(relearn_ctx *c, relearn_update_stats *stats)
{
    if (!c || !stats) return RELEARN_ERR_INVALID_ARG;
    if (!c->stats_valid && !c->length_ran)
        return fail(c, RELEARN_ERR_STATE, "no connectivity update has run");
    DeviceGuard g(c->device);
    relearn_status s = sync(c);
    int64_t h[16];
    CK(cudaMemcpy(h, c->d_i64, sizeof(h), cudaMemcpyDeviceToHost), "stats copy");
    memset(stats, 0, sizeof(*stats));
    stats->searches = h[I64_Q];
    stats->failed = h[I64_FAILED];
    stats->requests_declined = h[I64_DECLINED];
    stats->formed = h[I64_FORMED];
    stats->synapses = h[I64_NSYN];
    stats->searches_total = h[I64_Q_TOTAL];
    stats->evals_total = h[I64_EVALS_TOTAL];
    stats->walk_steps_total = h[I64_STEPS_TOTAL];
    stats->length_evals_total = h[I64_LEN_EVALS];
    if (c->timed) {
        cudaEventElapsedTime(&stats->ms_reduce, c->ev[0], c->ev[1]);
        cudaEventElapsedTime(&stats->ms_search, c->ev[1], c->ev[3]);
        cudaEventElapsedTime(&stats->ms_search_kernel, c->ev[2], c->ev[3]);
        cudaEventElapsedTime(&stats->ms_accept, c->ev[3], c->ev[4]);
        cudaEventElapsedTime(&stats->ms_apply, c->ev[4], c->ev[5]);
        cudaEventElapsedTime(&stats->ms_total, c->ev[0], c->ev[5]);
    }
    return s;
}

relearn_status relearn_collect_search_times(relearn_ctx *c, double *total_ms, int64_t *launches)
{
    if (!c || !total_ms || !launches) return RELEARN_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    relearn_status s = sync(c);
    double tot = 0.0;
    for (int k = 0; k < c->nkev; ++k) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, c->kev[k][0], c->kev[k][1]), "event time");
        tot += ms;
    }
    *total_ms = tot;
    *launches = c->nkev;
    c->nkev = 0;
    return s;
}

relearn_status relearn_launch_count(int64_t *count)
{
    if (!count) return RELEARN_ERR_INVALID_ARG;
    *count = g_launches.load(std::memory_order_relaxed);
    return RELEARN_OK;
}

relearn_status relearn_last_error(relearn_ctx *c, const char **msg)
{
    if (!c) {
        if (msg) *msg = "NULL context";
        return RELEARN_ERR_INVALID_ARG;
    }
    DeviceGuard g(c->device);
    relearn_status s = sync(c);
    if (s == RELEARN_OK) s = c->host_error;
    if (msg) *msg = s == RELEARN_OK ? "" : c->msg;
    c->host_error = RELEARN_OK;
    return s;
}

} // extern "C"
