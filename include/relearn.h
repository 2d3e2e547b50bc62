/*
 * relearn.h -- C ABI of librelearn.so: the Barnes-Hut connectivity update of the
 * Model of Structural Plasticity (MSP) on one GB300 (sm_103a).
 *
 * Paper: "I Like To Move It -- Computation Instead of Data in the Brain",
 * arXiv 2509.26193. Sec. III-A defines the three sub-steps of a connectivity
 * update (deletion, formation search, acceptance); Sec. III-B defines the
 * octree, its bottom-up update and the Barnes-Hut partner search with restarts.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller unless marked
 *     "host". The context owns all of its internal scratch (allocated once, in
 *     relearn_create). Neuron ids are 0 .. n-1 in the caller's order.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All work is enqueued on it; calls return before the GPU finishes unless a
 *     host output (stats, get_*) is requested, which synchronises the stream.
 *   - Argument and state errors are detected on the host and returned
 *     immediately; nothing is enqueued then. Device-side conditions (capacity
 *     overflow) are recorded in a device status word and returned by the next
 *     synchronising call (relearn_last_error, relearn_get_*, or an update with
 *     stats). The library never aborts the process and never traps the GPU.
 *   - A context is bound to one device and is not thread-safe; calls on one
 *     context must be issued from one host thread, on streams the caller keeps
 *     ordered.
 *   - Graph capture: build, update (stats NULL), deletion (broken NULL), delivery and
 *     the mean-length pair enqueue only device work with device-side counts, so a
 *     sequence of them can be captured into a CUDA graph and replayed. An update
 *     captured with RELEARN_FLAG_TIMING puts its phase events into the graph as
 *     event-record nodes: after a replay, relearn_get_last_stats returns that
 *     replay's phase times (of the last update captured with the flag). The context's host-side bookkeeping (whether the store is in canonical
 *     order, which diagnostics are valid) follows the captured calls, not the replays:
 *     a replayed sequence must end in the same store state its capture ended in (e.g.
 *     end with a deletion, or call relearn_get_synapses only after direct calls).
 */
#ifndef RELEARN_H
#define RELEARN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RELEARN_OK = 0,
    RELEARN_ERR_INVALID_ARG = 1, /* NULL where required, n out of range, sigma <= 0, theta < 0 */
    RELEARN_ERR_CUDA = 2,        /* a CUDA runtime call failed; see relearn_last_error */
    RELEARN_ERR_OOM = 3,         /* device allocation failed in relearn_create */
    RELEARN_ERR_CAPACITY = 4,    /* searches or synapses exceeded the context's capacity */
    RELEARN_ERR_TIMEOUT = 5,     /* a bounded device wait gave up (bottom-up update) */
    RELEARN_ERR_STATE = 6        /* call out of order (e.g. update before build) */
} relearn_status;

typedef struct relearn_ctx relearn_ctx;

/* Parameters of one connectivity update or deletion pass.
 *   sigma     kernel width (same length unit as the positions), > 0. The attraction of a
 *             candidate node with `count` vacant dendritic elements at distance d is
 *             count * exp(-d^2 / sigma^2).
 *   theta     Barnes-Hut acceptance parameter, >= 0: a node is accepted when its cell
 *             length (longest edge) divided by the distance to its centroid is < theta
 *             (Sec. II; theta = 0 gives the exact O(n^2) draw).
 *   seed      key of every Philox4x32-10 draw.
 *   step      update index (< 2^32), part of every Philox counter.
 *   flags     RELEARN_FLAG_* bits.
 *   search_group  tuning only: how many source neurons walk the octree together in the
 *             search kernel. The requests do not depend on it, except that one source per
 *             warp (2) sums its candidates in another association, so its draws may
 *             differ from the others' within rounding of a cumulative boundary.
 *             1, 8, 16 or 32 = a fixed width;
 *             2 = one source per warp, its frontier walk shared out over the 32 lanes;
 *             0 = the default: one source per warp when the update has at most 9 sources
 *             per resident warp of the union kernel, else unions chosen per warp: its 32
 *             sources (Morton order) cut at the boundaries of cells of depth 2 when at
 *             least 30 % of the neurons search, else of depth 4, one union per piece;
 *             1000 + 100 * d + r (d = 0..10, r = 0..10, r unused) = the default with the
 *             pieces cut at the boundaries of depth-d cells;
 *             3000 + f (f = 0..999) = the default with one source per warp for updates of
 *             at most f * 1024 sources.
 *   net_sigma, net_theta  device float[num_networks] or NULL (updates only): per-network
 *             sigma and theta of a batched build (relearn_build_octree_batch), replacing the
 *             scalars for network b. Values are checked on the device: a sigma that is not
 *             in (0, 3e38) or a theta not in [0, 3e38) sets INVALID_ARG in the device status
 *             and the update applies nothing. */
typedef struct {
    float sigma;
    float theta;
    uint64_t seed;
    uint64_t step;
    uint32_t flags;
    uint32_t search_group;
    const float *net_sigma;
    const float *net_theta;
} relearn_params;

/* Record per-search diagnostics (root-frontier ln S, node evaluations, restarts),
 * readable with relearn_get_search_diag. Costs a little extra memory traffic. */
#define RELEARN_FLAG_DIAG 1u
/* Record CUDA events around the phases of the update (stream-ordered, no
 * synchronisation); read them later with relearn_get_last_stats and
 * relearn_collect_search_times. */
#define RELEARN_FLAG_TIMING 2u
/* Two-phase search: a search whose first draw (on the root frontier) is an inner node is
 * queued; the queue is sorted by that node (pre-order = subtree order) and finished by a
 * separate kernel in which neighbouring threads restart inside the same subtree. Results
 * are bit-identical to the default (restarts finished inline by the lane that drew). */
#define RELEARN_FLAG_REGROUP 4u
/* Count node evaluations and walk steps into evals_total / walk_steps_total of
 * relearn_update_stats (RELEARN_FLAG_DIAG counts as well). Counting costs about one
 * instruction per step of the search walks (a few per cent of the search time), so
 * updates run without either flag add nothing to those totals. */
#define RELEARN_FLAG_COUNT 8u

/* Host-side summary of one update (filled when a stats pointer is passed; this
 * synchronises the stream). Times are CUDA-event milliseconds. */
typedef struct {
    int64_t searches;          /* Q = sum of vacant axonal elements at the start */
    int64_t failed;            /* searches with zero total attraction */
    int64_t requests_declined; /* requests refused by over-requested targets */
    int64_t formed;            /* synapses formed */
    int64_t synapses;          /* synapses stored after the update */
    float ms_reduce;        /* bottom-up octree update */
    float ms_search;        /* query setup + search kernel */
    float ms_search_kernel; /* the search kernel alone */
    float ms_accept, ms_apply, ms_total;
    int32_t reserved;
    int64_t searches_total;     /* searches of every update since the context was created */
    int64_t evals_total;        /* node evaluations (count > 0) of the searches of updates run
                                   with RELEARN_FLAG_COUNT or RELEARN_FLAG_DIAG: the work of the
                                   search, one per frontier candidate */
    int64_t walk_steps_total;   /* node visits of the grouped root-frontier walks (one node load
                                   per group of source neurons), for the same updates */
    int64_t length_evals_total; /* frontier candidates visited by the mean-length forward and
                                   backward kernels since the context was created */
} relearn_update_stats;

/* Create a context on CUDA device `device` that can hold up to max_neurons
 * neurons, max_synapses synapses and max_searches searches per update
 * (0 = 8 * max_neurons). Allocates all device scratch now.
 * Returns RELEARN_ERR_OOM if the allocation fails (nothing is leaked). */
relearn_status relearn_create(relearn_ctx **out, int device, int64_t max_neurons,
                              int64_t max_synapses, int64_t max_searches);

/* As relearn_create, for batched builds of up to max_networks independent networks
 * (relearn_build_octree_batch); max_networks in 1 .. RELEARN_MAX_NETWORKS. The batched
 * form has no counterpart in the paper, which updates one network: it packs many small
 * networks into one build and one search launch so the GPU is filled. */
#define RELEARN_MAX_NETWORKS 65536
relearn_status relearn_create_batched(relearn_ctx **out, int device, int64_t max_neurons,
                                      int64_t max_synapses, int64_t max_searches,
                                      int32_t max_networks);

/* Free the context and all of its device memory (synchronises the device). NULL is ok. */
relearn_status relearn_destroy(relearn_ctx *ctx);

/* Build the spatial octree over n neurons (Sec. III-B "Spatial octree").
 *   x, y, z     device float[n], positions (SoA). Copied into the context in
 *               Morton order; the caller may free them afterwards.
 *   vac_de      device int32[n] or NULL: when given, the bottom-up update also runs, so
 *               the tree is ready for inspection (relearn_get_tree).
 *   box_lo3/hi3 host float[3] each, or both NULL: the domain box. NULL = the bounding box
 *               of the positions. Positions outside a given box are clamped to it.
 * Steps: 30-bit Morton codes (10 bits per axis, FP32 quantisation
 * floor(((x - lo) * (1/(hi - lo))) * 1024) clamped to 0..1023), a stable radix sort of
 * (code, id), and the compressed octree: the root, every cell with >= 2 non-empty
 * children, every depth-10 cell with >= 2 neurons (a bucket) and one leaf per neuron, in
 * pre-order with skip links. The topology stays valid until the next build.
 * Errors: INVALID_ARG for n < 1, n > max_neurons, NULL positions. */
relearn_status relearn_build_octree(relearn_ctx *ctx, int64_t n, const float *x, const float *y,
                                    const float *z, const int32_t *vac_de, const float *box_lo3,
                                    const float *box_hi3, void *stream);

/* Build one octree per network for num_networks independent networks in one pass (no
 * counterpart in the paper; each network is the single network of Sec. III-B).
 *   offsets   host int64[num_networks + 1]: network b holds neuron ids offsets[b] ..
 *             offsets[b + 1] - 1; offsets[0] = 0, strictly increasing (no empty network),
 *             offsets[num_networks] = n <= max_neurons. The offsets are staged in pinned
 *             memory owned by the context; a build captured into a CUDA graph reads the
 *             offsets of the latest build call when the graph runs.
 *   x, y, z, vac_de  as relearn_build_octree, over all n neurons.
 * Each network's domain is the bounding box of its own positions. Every later call works
 * on all networks at once: an update searches each neuron's own network only (a network's
 * tree is its own subtree, so no synapse crosses networks), with per-network sigma/theta
 * from relearn_params.net_sigma/net_theta; Philox counters use the global neuron ids.
 * Errors: INVALID_ARG for bad offsets, num_networks outside 1 .. the context's
 * max_networks, NULL positions. */
relearn_status relearn_build_octree_batch(relearn_ctx *ctx, int32_t num_networks,
                                          const int64_t *offsets, const float *x, const float *y,
                                          const float *z, const int32_t *vac_de, void *stream);

/* One connectivity update (Sec. III-A "Update of synapses", formation sub-phase, with the
 * Barnes-Hut search of Sec. III-B):
 *   1. bottom-up update of the octree from vac_de (counts, count-weighted centroids);
 *   2. one search per vacant axonal element (neuron i, element e < vac_ax[i]) from the
 *      root: rejected nodes are replaced by their children, one accepted node is drawn
 *      with probability proportional to its attraction (draw word
 *      Philox4x32-10({i, step, (e << 8) | depth(start), 0}, seed).x), an inner node
 *      restarts the search from itself, a leaf becomes the request target; the searching
 *      neuron's own leaf has attraction 0; zero total attraction = failed search;
 *   3. acceptance: a target with more requests than vac_de accepts the vac_de requests with
 *      the smallest priority Philox4x32-10({i, step, (e << 8) | 0xFF, 1}, seed).x
 *      (ties by source id, then element);
 *   4. apply: accepted requests decrement vac_ax[src] and vac_de[tgt] and add synapse
 *      (src, tgt, sign = type[src] ? -1 : +1) to the context's store.
 *   params    host pointer.
 *   vac_ax    device int32[n], in/out.  vac_de  device int32[n], in/out (negative = 0).
 *   type      device uint8[n]: 0 excitatory, 1 inhibitory.
 *   stats     host pointer or NULL; non-NULL synchronises the stream and fills it.
 * Errors: STATE before a build; INVALID_ARG for bad params or NULL arrays; CAPACITY
 * (device status) if Q > max_searches or the store would overflow -- then nothing is
 * applied. */
relearn_status relearn_update_connectivity(relearn_ctx *ctx, const relearn_params *params,
                                           int32_t *vac_ax, int32_t *vac_de,
                                           const uint8_t *type, relearn_update_stats *stats,
                                           void *stream);

/* Typed dendrite pools (a variant of the update above): every neuron has vacant excitatory
 * (vac_de_exc) and inhibitory (vac_de_inh) dendritic elements; an excitatory axon (type 0)
 * searches a tree of the excitatory pool only, an inhibitory axon (type 1) the inhibitory
 * pool, and each pool of a target accepts only the requests made to it (the request's cell
 * type, Sec. III-B, selects the pool). The pools never interact, so this is the update
 * above once per pool on the same topology, restricted to that pool's axons, with the same
 * Philox counters; vac_ax and both pools are updated in place, synapse sign = source type.
 * relearn_get_requests / relearn_get_search_diag then describe the inhibitory pass.
 * stats (host or NULL) sums the two passes. Errors: as relearn_update_connectivity; the two
 * pool arrays must be different. */
relearn_status relearn_update_connectivity_typed(relearn_ctx *ctx, const relearn_params *params,
                                                 int32_t *vac_ax, int32_t *vac_de_exc,
                                                 int32_t *vac_de_inh, const uint8_t *type,
                                                 relearn_update_stats *stats, void *stream);

/* Testing hook for the bounded waits of the update's query setup (a single-pass scan
 * in which each tile of 4096 neurons waits for the sums its predecessors publish): in
 * the next update of this context the scan tile `tile` publishes nothing, so the tiles
 * after it wait until their bound runs out (2^16 rounds of reads, tens of
 * milliseconds). That update then reports RELEARN_ERR_TIMEOUT at its next
 * synchronising call and applies nothing; the context stays usable. tile < 0 clears
 * the hook. Errors: INVALID_ARG for NULL. */
relearn_status relearn_debug_stall_scan(relearn_ctx *ctx, int64_t tile);

/* Deletion pass (Sec. III-A "Update of synapses", first sub-phase).
 *   retract_ax, retract_de  device int32[n] (>= 0): elements each neuron retracts.
 *   vac_ax, vac_de          device int32[n], in/out.
 * Vacant elements are retracted first. The remainder (capped by the neuron's bound
 * elements) breaks that many of its synapses on the same side, chosen by the smallest
 * priority Philox4x32-10({neuron, step, slot, 2 (axonal) | 3 (dendritic)}, seed).x over the
 * slots of its out-row (ordered by target) or in-row (ordered by source); ties by slot. A
 * broken synapse gives its partner one vacant element, unless both ends picked it.
 * If `broken` (host) is non-NULL the stream is synchronised and the count written. */
relearn_status relearn_delete_synapses(relearn_ctx *ctx, const relearn_params *params,
                                       const int32_t *retract_ax, const int32_t *retract_de,
                                       int32_t *vac_ax, int32_t *vac_de, int64_t *broken,
                                       void *stream);

/* Spike delivery over the synapse store (Sec. III-A "Update of electrical activity"):
 *   input[t] = sum over synapses s -> t of sign(s) * spiked[s]   (duplicates count).
 *   spiked  device uint8[n] (0/1).  input  device int32[n], written. */
relearn_status relearn_deliver_spikes(relearn_ctx *ctx, const uint8_t *spiked, int32_t *input,
                                      void *stream);

/* Firing-rate-approximated spike delivery (Sec. IV-B, "Approximation of firing rates"):
 * instead of receiving spikes, neuron t decides once per step and per presynaptic
 * neuron s whether s spiked, from s's firing rate and a PRNG:
 *   spiked(s, t) = Philox4x32-10({s, t, step, 4}, seed).x < rate[s] * 2^32,
 *   input[t] = sum over synapses s -> t of sign(s) * spiked(s, t)   (duplicates count).
 *   rate   device float[n], probability of a spike per step (values <= 0 never, >= 1
 *          always spike).  input  device int32[n], written.  step < 2^32. */
relearn_status relearn_deliver_rates(relearn_ctx *ctx, const float *rate, uint64_t seed,
                                     uint64_t step, int32_t *input, void *stream);

/* Differentiable form (no counterpart in the paper, which only samples partners): the
 * expected synapse length over the root frontier, a smooth field of sigma and the
 * positions. For a source i with m_i = vac_ax[i] > 0, F_i = the candidates of its first
 * draw (the search of relearn_update_connectivity from the root, own leaf excluded);
 * with D_ik = |x_i - c_k|^2, d_ik = sqrt(D_ik), a_ik = N_k exp(-D_ik / sigma^2):
 *   l_i = sum_k a_ik d_ik / sum_k a_ik,   mean = sum_i m_i l_i / sum_i m_i,
 * the sums over the sources whose total attraction is > 0.
 *   params  sigma and theta (or net_sigma[0] / net_theta[0], device); seed/step unused.
 *   vac_ax  device int32[n]: the weights m.  vac_de  device int32[n]: N_k and the centroid
 *           weights (the bottom-up update runs here, Sec. III-B).
 *   ell     device float[n] or NULL: l_i by neuron id, NaN where excluded.
 *   mean    device double, written (NaN when no source is included).
 * FP32 attractions with compensated sums, l and the normaliser in FP64. Needs a
 * single-network build (STATE otherwise). */
relearn_status relearn_mean_length(relearn_ctx *ctx, const relearn_params *params,
                                   const int32_t *vac_ax, const int32_t *vac_de, float *ell,
                                   double *mean, void *stream);

/* Adjoint of relearn_mean_length (call it right after its forward, same vac_ax and vac_de;
 * STATE if a build or an update came in between). The acceptance criterion and the tree
 * topology are piecewise constant and contribute nothing:
 *   dl_i/dsigma = (2 / sigma^3) sum_k q_ik (d_ik - l_i) (D_ik - Dbar_i),  q = a / S,
 *   dl_i/dc_k = q_ik r_ik (2 (d_ik - l_i) / sigma^2 - 1 / d_ik),  r = x_i - c_k,
 *   dl_i/dx_i = -sum_k dl_i/dc_k,  dc_k/dx_j = vac_de[j] / N_k for each neuron j in cell k.
 *   grad_mean  device double or NULL (= 1): the upstream gradient of mean.
 *   gx, gy, gz device float[n], written: d(grad_mean * mean)/d(position), by neuron id.
 *   gsigma     device double or NULL, written: d(grad_mean * mean)/d sigma.
 * Attractions are recomputed, not stored; the centroid adjoints are accumulated per
 * node with FP32 vector atomics (order not fixed: the gradient is reproducible to
 * FP32 rounding, not bit for bit). */
relearn_status relearn_mean_length_backward(relearn_ctx *ctx, const int32_t *vac_ax,
                                            const int32_t *vac_de, const double *grad_mean,
                                            float *gx, float *gy, float *gz, double *gsigma,
                                            void *stream);

/* Copy the synapse store to host arrays in canonical order (by source, then target).
 * `count` (host) receives the number stored; src/tgt/sign may be NULL to query only the
 * count, else they must hold `capacity` entries (INVALID_ARG if too small).
 * Synchronises the context's stream and returns any pending device status. */
relearn_status relearn_get_synapses(relearn_ctx *ctx, int64_t capacity, int64_t *count,
                                    int32_t *src, int32_t *tgt, int8_t *sign);

/* Replace the synapse store from host arrays (any order; it is canonicalised).
 * Used for checkpoint/resume together with the vacancy arrays. Synchronous. */
relearn_status relearn_set_synapses(relearn_ctx *ctx, int64_t count, const int32_t *src,
                                    const int32_t *tgt, const int8_t *sign);

/* Copy the last update's requests to host arrays, in canonical query order (neuron id,
 * then element): tgt (-1 = failed search) and accept (0/1). `count` receives Q.
 * Synchronous. */
relearn_status relearn_get_requests(relearn_ctx *ctx, int64_t capacity, int64_t *count,
                                    int32_t *tgt, uint8_t *accept);

/* Per-search diagnostics of the last update run with RELEARN_FLAG_DIAG, canonical query
 * order: ln_s0 (natural log of the root frontier's total attraction, -inf when zero),
 * evals (node evaluations with count > 0 over all draws), restarts. Synchronous. */
relearn_status relearn_get_search_diag(relearn_ctx *ctx, int64_t capacity, int64_t *count,
                                       double *ln_s0, int32_t *evals, int32_t *restarts);

/* Copy the current octree to host arrays, pre-order (parent first, children in Morton
 * order). Per node: depth (0..10; leaves report the depth of their parent + 1, capped at
 * 11 inside buckets), first (position of its first neuron in Morton order), size (neurons),
 * is_leaf, neuron (id for leaves, -1 otherwise), count (vacant dendritic elements) and
 * centroid cx/cy/cz (float, 0 when count == 0). Any output may be NULL. `perm` (host
 * int32[n] or NULL) receives the neuron ids in Morton order. Synchronous. */
relearn_status relearn_get_tree(relearn_ctx *ctx, int64_t capacity, int64_t *num_nodes,
                                int32_t *depth, int32_t *first, int32_t *size, int32_t *is_leaf,
                                int32_t *neuron, int32_t *count, float *cx, float *cy, float *cz,
                                int32_t *perm);

/* Device Philox4x32-10 over `count` blocks (the generator the kernels use): ctr is
 * device uint32[4*count], key device uint32[2*count], out device uint32[4*count]. */
relearn_status relearn_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                                     int64_t count, void *stream);

/* Counters and (when the update ran with RELEARN_FLAG_TIMING or a stats pointer) phase
 * times of the last connectivity update. Synchronises the context's stream. Times are 0
 * when no events were recorded. */
relearn_status relearn_get_last_stats(relearn_ctx *ctx, relearn_update_stats *stats);

/* Sum of the search-kernel durations (CUDA events, ms) of the updates run with
 * RELEARN_FLAG_TIMING since the previous call (up to 64), and how many there were.
 * Synchronises the context's stream; resets the record. Host pointers. */
relearn_status relearn_collect_search_times(relearn_ctx *ctx, double *total_ms, int64_t *launches);

/* Total number of CUDA kernels this library has launched in the process (all contexts).
 * `count` is a host pointer. Never fails for a non-NULL pointer. */
relearn_status relearn_launch_count(int64_t *count);

/* Measurement probes for the roofline denominators (no counterpart in the paper; used by
 * the benchmark to measure, on the GPU at hand, the rates that bound the search):
 *   kind 1  FP32 FMA issue (independent chains of fma.rn.f32), *ops = FMAs;
 *   kind 2  special-function unit ex2.approx.ftz.f32, *ops = ex2 evaluations;
 *   kind 3  L2 read bandwidth: `iters` passes of 16-byte L2-only loads over buf,
 *           *ops = bytes read (buf 16-byte aligned, buf_len >= 4 floats);
 *   kind 4  packed FP32 FMA (fma.rn.f32x2), *ops = FMAs (two per instruction).
 * One launch of about 4 blocks of 256 threads per SM on `stream`; the caller times it.
 * buf is a caller-owned device float[buf_len]; kinds 1, 2 and 4 overwrite up to one
 * element per thread, kind 3 only reads it. `ops` is a host pointer written before the
 * launch. Errors: INVALID_ARG for iters < 1, a NULL pointer, an unknown kind or a bad
 * kind-3 buffer (nothing launched); CUDA when a launch error is already pending (left
 * pending) or the launch fails. */
relearn_status relearn_peak_probe(int32_t kind, int64_t iters, float *buf, int64_t buf_len,
                                  int64_t *ops, void *stream);

/* Allocation-free Morton ordering, for callers that must not allocate device memory
 * (no counterpart in the paper; it exists for users of this library): the neurons'
 * 30-bit Morton codes (same quantisation as relearn_build_octree) and their stable
 * order by (code, id), without a context and without any cudaMalloc/cudaFree.
 *   n            1 .. RELEARN_NOALLOC_MAX_NEURONS; larger n returns RELEARN_ERR_CAPACITY.
 *   x, y, z      device float[n], positions.
 *   box_lo3/hi3  host float[3] each, or both NULL (= bounding box of the positions).
 *   codes        device uint32[n], out: the codes in ascending order.
 *   perm         device int32[n], out: perm[k] = id of the neuron with the k-th code
 *                (ties by id), the same order relearn_get_tree reports.
 * The sort's scratch is one static device array of about 8.5 MB per GPU, held until the
 * process exits. Every call looks up that array's device address on the current device
 * (a lookup, no allocation); the first call on each device also reads its SM count and
 * may make the driver load this library's kernels there, so make that first call before
 * any stream capture. All calls on a device share the array: calls whose GPU work
 * overlaps race and give wrong results, so order them on one stream (or otherwise).
 * A launch error left pending by earlier, unrelated work makes the call return
 * RELEARN_ERR_CUDA at once, launching nothing and leaving that error pending for its
 * owner. Asynchronous on `stream`. */
#define RELEARN_NOALLOC_MAX_NEURONS (1 << 20)
relearn_status relearn_morton_order_noalloc(int64_t n, const float *x, const float *y,
                                            const float *z, const float *box_lo3,
                                            const float *box_hi3, uint32_t *codes, int32_t *perm,
                                            void *stream);

/* Synchronise the context's last stream, fold the device status word into the result and
 * return it; *msg (host, may be NULL) points at a static description of the last error.
 * Clears the stored error. */
relearn_status relearn_last_error(relearn_ctx *ctx, const char **msg);

#ifdef __cplusplus
}
#endif

#endif /* RELEARN_H */
