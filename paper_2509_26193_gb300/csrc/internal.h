// Host-side internals of librelearn: the context and the kernel launchers that
// the translation units share. Not installed; the public ABI is relearn.h.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/relearn.h"
#include "device.cuh"

namespace rl {

// Scratch of the device-wide single-pass exclusive scan.
struct ScanScratch {
    int64_t *block_sums = nullptr; // [4 * max_blocks]: tile sums, then inclusive prefixes
                                   // (pairs of them for a pair scan)
    int32_t *flags = nullptr;      // [max_blocks + 3]: ticket, abort, blocks done, tile
                                   // states; zero between scans
    int32_t *status = nullptr;     // device status word for a wait that ran out (or NULL)
    int64_t max_blocks = 0;
    int64_t grid_cap = 1 << 30;    // blocks a scan launches at most (the resident ones)
};

// Scratch of the LSD radix sort (per-block digit histograms, digit-major).
struct SortScratch {
    int32_t *hist = nullptr;      // [256 * max_blocks]
    int64_t max_blocks = 0;
    ScanScratch scan;
};

// Per-build geometry, device resident.
struct Geom {
    float lo[3], hi[3], inv[3];
    float pad;
    double ext;      // longest edge of the domain box
    double fx_lo[3]; // origin of the fixed-point positions (below every position and lo)
    double fx_scale; // 2^k: positions are held as round((x - fx_lo) * 2^k) < 2^30
    double fx_inv;   // 2^-k
};

// Per-update search constants computed on the device from Geom and params.
struct SearchConst {
    uint32_t thr0; // bits of (root cell length / theta)^2 (FLT_MAX for theta = 0)
    float k2;      // log2(e) / sigma^2
    float sigma;
    float pad;
};

} // namespace rl

struct relearn_ctx {
    int device = 0;
    int num_sms = 0;
    // resident blocks per SM: [2 * batched + diagnostics][union, split]
    int search_occ[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    int split_occ[2][33] = {};  // split kernel blocks per SM, by network kind and capacity / 32
    int64_t max_neurons = 0, max_synapses = 0, max_searches = 0, max_nodes = 0;
    int32_t max_nets = 1; // networks one build may hold
    int32_t num_nets = 1; // networks in the current tree
    cudaStream_t last_stream = nullptr;
    bool built = false;
    int64_t n = 0; // neurons in the current tree
    relearn_status host_error = RELEARN_OK;
    char msg[256] = {0};

    // ---- device scalars (one block, see api.cu for the slot map)
    int32_t *d_status = nullptr;   // first device error code
    int64_t *d_i64 = nullptr;      // [16] counters and totals
    int32_t *d_i32 = nullptr;      // [16] element counts used as kernel bounds
    rl::Geom *d_geom = nullptr;      // [max_nets]
    rl::SearchConst *d_sc = nullptr; // [max_nets]

    // ---- networks: b holds neurons off[b] .. off[b + 1] - 1 (ids and Morton positions)
    int64_t *d_off = nullptr;     // [max_nets + 1]
    int64_t *h_off = nullptr;     // [max_nets + 1] pinned staging of the offsets
    cudaEvent_t off_ev = nullptr; // the last copy out of h_off
    uint32_t *d_ord = nullptr;    // [6 * max_nets] bounding boxes (ordered-int min, max)
    int32_t *d_root = nullptr;    // [max_nets] root node of each network
    int32_t *d_net = nullptr;     // [n] network of each Morton position (max_nets > 1)
    uint64_t *d_nkey = nullptr, *d_nkey_alt = nullptr; // [n] (network, code) sort keys

    // ---- tree (per build)
    uint32_t *d_codes = nullptr, *d_codes_alt = nullptr; // [n]
    int32_t *d_perm = nullptr, *d_perm_alt = nullptr;    // Morton position -> neuron id
    float4 *d_pos = nullptr;                             // positions in Morton order
    int4 *d_posq = nullptr;                              // fixed-point positions, Morton order
    uint32_t *d_mask = nullptr;                          // [n] depths of nodes starting here
    int32_t *d_base = nullptr;                           // [n + 1] pre-order index of position
    rl::Node *d_nodes = nullptr;                         // [max_nodes]
    int32_t *d_parent = nullptr;                         // [max_nodes] (get_tree)
    int32_t *d_nsize = nullptr;                          // [max_nodes] neurons in the node's cell
    int32_t *d_leaf = nullptr;                           // [n] leaf node of each position
    double *d_acc = nullptr;  // bottom-up update: int64 x 4 prefix and tile sums
    int64_t debug_stall_tile = -1; // relearn_debug_stall_scan: next update only

    // ---- queries and requests (per update)
    int32_t *d_cnt = nullptr;       // [n + 1] scratch counts
    int32_t *d_act_off = nullptr;   // [n + 1] rank of each Morton position among active sources
    int32_t *d_qoff_o = nullptr;    // [n + 1] request offsets, id order
    int32_t *d_act_src = nullptr;   // [n] Morton positions of neurons with vacant axons
    int32_t *d_req_src = nullptr;   // [max_searches] canonical order
    int32_t *d_req_elem = nullptr;  // [max_searches]
    int32_t *d_req_tgt = nullptr;   // [max_searches]
    uint8_t *d_req_acc = nullptr;   // [max_searches]
    uint32_t *d_req_prio = nullptr; // [max_searches]
    uint64_t *d_bucket = nullptr;   // [max_searches] request keys grouped by target
    int32_t *d_tcnt = nullptr, *d_toff = nullptr; // [n + 1]
    int32_t *d_newpos = nullptr;    // [max_searches + 1]
    uint32_t *d_rq_key = nullptr, *d_rq_key_alt = nullptr; // [max_searches] deferred restarts
    int32_t *d_rq_val = nullptr, *d_rq_val_alt = nullptr;
    int32_t *d_rq_out = nullptr, *d_rq_src = nullptr;
    double *d_diag_lns = nullptr;   // [max_searches] (diag only)
    int32_t *d_diag_evals = nullptr, *d_diag_restarts = nullptr;

    // ---- synapse store (canonical by (src, tgt)) and its views
    int32_t *d_syn_src = nullptr, *d_syn_tgt = nullptr; // [max_synapses]
    int8_t *d_syn_sign = nullptr;
    uint64_t *d_key = nullptr, *d_key_alt = nullptr;    // [max_synapses] sort keys
    int32_t *d_val = nullptr, *d_val_alt = nullptr;     // [max_synapses]
    uint32_t *d_key32 = nullptr, *d_key32_alt = nullptr;
    int32_t *d_out_ptr = nullptr, *d_in_ptr = nullptr;  // [max_neurons + 1]
    int32_t *d_in_syn = nullptr;                        // [max_synapses]
    uint32_t *d_prio_ax = nullptr, *d_prio_de = nullptr; // [max_synapses]
    uint8_t *d_sel_ax = nullptr, *d_sel_de = nullptr;    // [max_synapses]
    int32_t *d_need_ax = nullptr, *d_need_de = nullptr;  // [max_neurons]
    int32_t *d_keep = nullptr;                           // [max_synapses + 1]

    // ---- differentiable form (expected synapse length, length.cu)
    float4 *d_lstate = nullptr; // [n] per source (Morton position): l, Dbar, 1/S, exponent shift
    double *d_lsum = nullptr;   // [4] sum m l, sum m (M), mean

    rl::ScanScratch scan;
    rl::SortScratch sort;

    cudaEvent_t ev[8] = {};
    bool timed = false; // the last update recorded its phase events
    cudaEvent_t kev[64][2] = {}; // search-kernel start/stop of timed updates
    int nkev = 0;
    bool diag_valid = false;
    bool stats_valid = false;
    bool canonical = true; // store sorted by (src, tgt) with stable views (else rows only)
    bool length_valid = false; // a mean-length forward ran since the last build or update
    bool length_ran = false;   // a mean-length forward ran at least once
};

// slots of d_i64 / d_i32
enum { I64_Q = 0, I64_FAILED, I64_DECLINED, I64_FORMED, I64_NSYN, I64_BROKEN, I64_SCAN_TOTAL,
       I64_NODES, I64_Q_TOTAL, I64_EVALS_TOTAL, I64_ACTIVE, I64_STEPS_TOTAL, I64_LEN_EVALS };
enum { I32_N = 0, I32_Q, I32_NSYN, I32_NEW, I32_NODES, I32_WORK, I32_ACTIVE, I32_RQ, I32_BASE };

namespace rl {

// Blocks for a grid-stride loop over n items: enough to cover n, at most 32 per SM.
inline unsigned grid_for(int64_t n, int threads, int num_sms)
{
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 32;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// api.cu --------------------------------------------------------------------
// Counts kernel launches made by the library (reported by relearn_launch_count).
void note_launch();

// scan.cu -------------------------------------------------------------------
// out[i] = sum(in[0 .. i)) for i < count; *total = sum(in[0 .. count)) (int64).
// count = d_count ? min(*d_count, max_n) : max_n. `out` may alias `in`.
cudaError_t scan_exclusive(const int32_t *in, int32_t *out, int64_t max_n, const int32_t *d_count,
                           int64_t *d_total, ScanScratch &s, cudaStream_t st);
int64_t scan_blocks_needed(int64_t max_n);
int64_t scan_grid_cap(int num_sms);
cudaError_t fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t st);

// sort.cu -------------------------------------------------------------------
// Stable LSD radix sort of (key, val) on bits [0, end_bit). Returns the buffer
// index holding the result (0: keys/vals, 1: the *_alt buffers) through *which.
cudaError_t radix_sort_u32(uint32_t *keys, uint32_t *keys_alt, int32_t *vals, int32_t *vals_alt,
                           int64_t max_n, const int32_t *d_count, int end_bit, SortScratch &s,
                           cudaStream_t st, int *which);
cudaError_t radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, int32_t *vals, int32_t *vals_alt,
                           int64_t max_n, const int32_t *d_count, int end_bit, SortScratch &s,
                           cudaStream_t st, int *which);
int64_t sort_blocks_needed(int64_t max_n);

// octree.cu -----------------------------------------------------------------
cudaError_t octree_build(relearn_ctx *c, int64_t n, int32_t B, const float *x, const float *y,
                         const float *z, const float *box_lo, const float *box_hi,
                         cudaStream_t st);
cudaError_t octree_reduce(relearn_ctx *c, const int32_t *vac_de, cudaStream_t st);

// search.cu -----------------------------------------------------------------
cudaError_t search_prepare(relearn_ctx *c, const relearn_params &p, const int32_t *vac_ax,
                           cudaStream_t st);
cudaError_t search_run(relearn_ctx *c, const relearn_params &p, const int32_t *vac_ax,
                       cudaStream_t st);

// length.cu -----------------------------------------------------------------
// Forward: per-source expected length over the root frontier and their mean.
cudaError_t length_forward(relearn_ctx *c, const int32_t *vac_ax, float *ell, double *mean,
                           cudaStream_t st);
// Adjoint of the mean with respect to sigma and the positions (after length_forward).
cudaError_t length_backward(relearn_ctx *c, const int32_t *vac_ax, const int32_t *vac_de,
                            const double *grad_mean, float *gx, float *gy, float *gz,
                            double *gsigma, cudaStream_t st);
// search.cu: per-network acceptance thresholds and kernel widths from params.
cudaError_t search_constants(relearn_ctx *c, const relearn_params &p, cudaStream_t st);

// synapses.cu ---------------------------------------------------------------
cudaError_t accept_requests(relearn_ctx *c, const relearn_params &p, const int32_t *vac_de,
                            cudaStream_t st);
cudaError_t apply_requests(relearn_ctx *c, int32_t *vac_ax, int32_t *vac_de, const uint8_t *type,
                           cudaStream_t st);
// Typed dendrite pools: out[i] = vac_ax[i] where type[i] == kind, else 0; and back.
cudaError_t select_type(relearn_ctx *c, const int32_t *vac_ax, const uint8_t *type, int kind,
                        int32_t *out, cudaStream_t st);
cudaError_t merge_type(relearn_ctx *c, const int32_t *part, const uint8_t *type, int kind,
                       int32_t *vac_ax, cudaStream_t st);
cudaError_t delete_synapses(relearn_ctx *c, const relearn_params &p, const int32_t *retract_ax,
                            const int32_t *retract_de, int32_t *vac_ax, int32_t *vac_de,
                            cudaStream_t st);
cudaError_t deliver_spikes(relearn_ctx *c, const uint8_t *spiked, int32_t *input,
                           cudaStream_t st);
cudaError_t canonicalise_store(relearn_ctx *c, cudaStream_t st);
cudaError_t deliver_rates(relearn_ctx *c, const float *rate, uint64_t seed, uint32_t step,
                          int32_t *input, cudaStream_t st);

} // namespace rl
