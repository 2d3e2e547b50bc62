/*
 * MSP connectivity-update oracle: plain, slow, FP64 CPU code written from the
 * paper "I Like To Move It -- Computation Instead of Data in the Brain"
 * (arXiv 2509.26193).
 *
 * THIS IS TEST INFRASTRUCTURE. It checks the CUDA path and shares no code with
 * it: no headers, no helpers, no tables. Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference leg load it; the product never does.
 *
 * Order follows the paper:
 *   Philox4x32-10 ........... Salmon et al., SC'11 (the paper only says that a PRNG
 *                             draws the partner, Sec. III-A "Update of synapses",
 *                             and that its stream is arbitrary, Sec. V-A)
 *   Morton quantisation ..... Sec. III-B "Division of the simulation domain"
 *   octree build ............ Sec. III-B "Spatial octree"
 *   bottom-up update ........ Sec. III-B "Division of work", first paragraph
 *   Barnes-Hut search ....... Sec. III-B "Division of work", second paragraph;
 *                             criterion and theta = 0 from Sec. II
 *   acceptance + apply ...... Sec. III-A "Update of synapses", second sub-phase
 *   deletion ................ Sec. III-A "Update of synapses", first sub-phase
 *   spike delivery .......... Sec. III-A "Update of electrical activity"
 *   firing-rate delivery .... Sec. IV-B "Approximation of firing rates"
 *   expected synapse length . the draw distribution of Sec. III-B as a smooth field,
 *                             with its gradient (not in the paper, R15)
 *
 * Readings where the paper is silent (restated at each function):
 *   R1  domain = bounding box of the positions unless a box is given (anisotropic cells)
 *   R2  cell "length" in the criterion = longest edge of the cell box
 *   R3  depth limit 10 (10 bits per axis); >= 2 neurons in one depth-10 cell form a
 *       bucket whose children are its neurons
 *   R4  accept iff len^2 < theta^2 * dist^2 (strict), dist = source to node centroid;
 *       single-neuron leaves are always accepted; the start node is always expanded
 *   R5  attraction = count * exp(-d^2 / sigma^2)
 *   R6  the searching neuron's own leaf has attraction 0
 *   R7  candidates in Morton (range-start) order; u = philox(...).x * 2^-32; the
 *       smallest k with u*S < C_k (C inclusive prefix sum) is drawn
 *   R8  zero total attraction: the search fails, the axonal element stays vacant
 *   R9  an over-requested target accepts the vac_de requests with the smallest
 *       Philox priority, ties by (source, element)
 *   R10 synapse sign = the source neuron's signal type (+1 excitatory, -1 inhibitory)
 *   R11 deletion retracts vacant elements first, then picks bound synapses by Philox
 *       priority per row slot; a synapse picked by both ends is broken once and
 *       returns no vacancy
 *   R12 duplicate (src, tgt) synapses are allowed and counted
 *   R13 firing-rate delivery: the receiver t decides once per step and per source s
 *       whether s spiked, w = philox({s, t, step, 4}, seed).x, spiked iff
 *       w < rate[s] * 2^32 (exact in FP64); every synapse s -> t then carries that spike
 *   R14 batched form (not in the paper): a tree may hold one network of a batch whose
 *       ids start at id_base; its search draws use the global id in the counter
 *   R15 differentiable form (not in the paper): the expected synapse length of a source
 *       is the attraction-weighted mean distance to the centroids of its root frontier
 *       (the first draw's candidates); its gradient treats the criterion and the tree
 *       topology as constant (see orc_mean_length)
 *   R16 typed dendrite pools (a variant; the paper's request carries a cell type,
 *       Sec. III-B): excitatory axons search excitatory dendritic elements, inhibitory
 *       axons inhibitory ones; composed from the functions here in oracle/__init__.py
 *
 * Every function here has a pin in the CPU test suite (tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_DEPTH 10

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11). Ten rounds of the 4x32 S-box with key schedule. */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static uint32_t philox_x(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint64_t seed)
{
    uint32_t c[4] = {w0, w1, w2, w3};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(c, k, o);
    return o[0];
}

/* ------------------------------------------------------------------------- */
/* Morton quantisation (Sec. III-B, "Division of the simulation domain": the
 * domain D is split into cells indexed along a space-filling curve).
 * An integer result decided by floating point: it is evaluated in FP32 exactly
 * as stated (round to nearest, no fused multiply-add):
 *     q = clamp(floor(((x - lo) * inv) * 1024), 0, 1023),  inv = 1 / (hi - lo)
 * and interleaved with the x bit lowest (bit 3k = x_k, 3k+1 = y_k, 3k+2 = z_k). */
/* ------------------------------------------------------------------------- */
static uint32_t quantise(float x, float lo, float inv)
{
    volatile float t = x - lo; /* volatile keeps every step a separate FP32 op */
    t = t * inv;
    t = t * 1024.0f;
    float c = fmaxf(t, 0.0f); /* NaN -> 0 */
    c = fminf(c, 1023.0f);
    return (uint32_t)c;
}

static float inverse_extent(float lo, float hi)
{
    volatile float ext = hi - lo;
    if (!(ext > 0.0f)) return 0.0f;
    volatile float one = 1.0f;
    return one / ext;
}

static uint32_t interleave(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint32_t code = 0;
    for (int b = 0; b < 10; ++b) {
        code |= ((qx >> b) & 1u) << (3 * b);
        code |= ((qy >> b) & 1u) << (3 * b + 1);
        code |= ((qz >> b) & 1u) << (3 * b + 2);
    }
    return code;
}

/* R1: the domain is the bounding box of the positions unless a box is given. */
static void domain_box(int64_t n, const float *x, const float *y, const float *z,
                       const float *box_lo, const float *box_hi, float lo[3], float hi[3])
{
    if (box_lo && box_hi) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = box_lo[a];
            hi[a] = box_hi[a];
        }
        return;
    }
    const float *p[3] = {x, y, z};
    for (int a = 0; a < 3; ++a) {
        float l = n > 0 ? p[a][0] : 0.0f, h = l;
        for (int64_t i = 1; i < n; ++i) {
            if (p[a][i] < l) l = p[a][i];
            if (p[a][i] > h) h = p[a][i];
        }
        lo[a] = l;
        hi[a] = h;
    }
}

void orc_morton(int64_t n, const float *x, const float *y, const float *z, const float *box_lo,
                const float *box_hi, uint32_t *codes, float *lo_out, float *hi_out)
{
    float lo[3], hi[3];
    domain_box(n, x, y, z, box_lo, box_hi, lo, hi);
    float inv[3];
    for (int a = 0; a < 3; ++a) inv[a] = inverse_extent(lo[a], hi[a]);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t qx = quantise(x[i], lo[0], inv[0]);
        uint32_t qy = quantise(y[i], lo[1], inv[1]);
        uint32_t qz = quantise(z[i], lo[2], inv[2]);
        codes[i] = interleave(qx, qy, qz);
    }
    if (lo_out && hi_out)
        for (int a = 0; a < 3; ++a) {
            lo_out[a] = lo[a];
            hi_out[a] = hi[a];
        }
}

/* ------------------------------------------------------------------------- */
/* Spatial octree (Sec. III-B "Spatial octree"): the root is the whole domain,
 * each cell splits into its eight octants, and subdivision stops when a cell
 * holds at most one neuron (R3: or at depth 10, where >= 2 neurons form a
 * bucket whose children are the neurons themselves, at depth 11).
 * A plain pointer tree: every cell with a neuron is a node, single-child
 * chains included. */
/* ------------------------------------------------------------------------- */
typedef struct {
    int depth;     /* 0..10 cells, 11 = member of a bucket */
    int leaf;      /* exactly one neuron */
    int neuron;    /* that neuron's id (leaf only) */
    int first;     /* range in canonical (Morton, then id) order */
    int size;      /* neurons in the cell */
    int nchild;    /* children are nodes child0 .. child0 + nchild - 1 */
    int child0;
    int parent;
    double count;  /* vacant dendritic elements (per update) */
    double sx, sy, sz; /* count-weighted position sums (per update) */
    double cx, cy, cz; /* weighted-average position; NaN when count == 0 */
} ONode;

typedef struct {
    int64_t n;
    int64_t id_base;                /* global id of neuron 0 (one network of a batch) */
    float lo[3], hi[3];
    double len2[ORC_MAX_DEPTH + 2]; /* (cell length)^2 per depth, R2 */
    double *px, *py, *pz;           /* positions as FP64 (exact copies of FP32 input) */
    uint32_t *qx, *qy, *qz;         /* quantised coordinates */
    int32_t *perm;                  /* canonical order of neuron ids */
    ONode *nodes;
    int64_t n_nodes, cap_nodes;
} OTree;

static int64_t new_node(OTree *T)
{
    if (T->n_nodes == T->cap_nodes) {
        T->cap_nodes = T->cap_nodes ? 2 * T->cap_nodes : 1024;
        T->nodes = (ONode *)realloc(T->nodes, (size_t)T->cap_nodes * sizeof(ONode));
    }
    ONode *v = &T->nodes[T->n_nodes];
    memset(v, 0, sizeof(*v));
    v->parent = -1;
    return T->n_nodes++;
}

static int cmp_int32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Subdivide cell v (holding perm[first .. first+size)) at depth `depth`. */
static void subdivide(OTree *T, int64_t v, int32_t *scratch)
{
    int depth = T->nodes[v].depth;
    int first = T->nodes[v].first, size = T->nodes[v].size;
    if (size <= 1) {
        T->nodes[v].leaf = 1;
        T->nodes[v].neuron = T->perm[first];
        return;
    }
    if (depth == ORC_MAX_DEPTH) {
        /* R3: bucket; its children are its neurons, ordered by id */
        qsort(T->perm + first, (size_t)size, sizeof(int32_t), cmp_int32);
        int64_t c0 = T->n_nodes;
        for (int k = 0; k < size; ++k) {
            int64_t c = new_node(T);
            ONode *nc = &T->nodes[c];
            nc->depth = ORC_MAX_DEPTH + 1;
            nc->leaf = 1;
            nc->neuron = T->perm[first + k];
            nc->first = first + k;
            nc->size = 1;
            nc->parent = (int)v;
        }
        T->nodes[v].child0 = (int)c0;
        T->nodes[v].nchild = size;
        return;
    }
    /* octant of each neuron at the next level: bit (9 - depth) of each axis */
    int shift = ORC_MAX_DEPTH - 1 - depth;
    int cnt[8] = {0};
    for (int k = 0; k < size; ++k) {
        int32_t i = T->perm[first + k];
        int oct = (int)(((T->qx[i] >> shift) & 1u) | (((T->qy[i] >> shift) & 1u) << 1) |
                        (((T->qz[i] >> shift) & 1u) << 2));
        cnt[oct]++;
    }
    int off[8], pos[8];
    off[0] = 0;
    for (int o = 1; o < 8; ++o) off[o] = off[o - 1] + cnt[o - 1];
    memcpy(pos, off, sizeof(pos));
    for (int k = 0; k < size; ++k) {
        int32_t i = T->perm[first + k];
        int oct = (int)(((T->qx[i] >> shift) & 1u) | (((T->qy[i] >> shift) & 1u) << 1) |
                        (((T->qz[i] >> shift) & 1u) << 2));
        scratch[pos[oct]++] = i;
    }
    memcpy(T->perm + first, scratch, (size_t)size * sizeof(int32_t));
    int nchild = 0;
    for (int o = 0; o < 8; ++o) nchild += cnt[o] > 0;
    int64_t c0 = T->n_nodes;
    for (int o = 0; o < 8; ++o) {
        if (!cnt[o]) continue;
        int64_t c = new_node(T);
        ONode *nc = &T->nodes[c];
        nc->depth = depth + 1;
        nc->first = first + off[o];
        nc->size = cnt[o];
        nc->parent = (int)v;
    }
    T->nodes[v].child0 = (int)c0;
    T->nodes[v].nchild = nchild;
    for (int k = 0; k < nchild; ++k) subdivide(T, c0 + k, scratch);
}

void *orc_tree_build(int64_t n, const float *x, const float *y, const float *z,
                     const float *box_lo, const float *box_hi)
{
    OTree *T = (OTree *)calloc(1, sizeof(OTree));
    T->n = n;
    domain_box(n, x, y, z, box_lo, box_hi, T->lo, T->hi);
    /* R2: cell length = longest edge of the cell box, halved per level */
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = (double)T->hi[a] - (double)T->lo[a];
        if (e > ext) ext = e;
    }
    for (int d = 0; d <= ORC_MAX_DEPTH + 1; ++d) {
        double len = ext / (double)(1u << d);
        T->len2[d] = len * len;
    }
    size_t nn = (size_t)(n > 0 ? n : 1);
    T->px = (double *)malloc(nn * sizeof(double));
    T->py = (double *)malloc(nn * sizeof(double));
    T->pz = (double *)malloc(nn * sizeof(double));
    T->qx = (uint32_t *)malloc(nn * sizeof(uint32_t));
    T->qy = (uint32_t *)malloc(nn * sizeof(uint32_t));
    T->qz = (uint32_t *)malloc(nn * sizeof(uint32_t));
    T->perm = (int32_t *)malloc(nn * sizeof(int32_t));
    float inv[3];
    for (int a = 0; a < 3; ++a) inv[a] = inverse_extent(T->lo[a], T->hi[a]);
    for (int64_t i = 0; i < n; ++i) {
        T->px[i] = x[i];
        T->py[i] = y[i];
        T->pz[i] = z[i];
        T->qx[i] = quantise(x[i], T->lo[0], inv[0]);
        T->qy[i] = quantise(y[i], T->lo[1], inv[1]);
        T->qz[i] = quantise(z[i], T->lo[2], inv[2]);
        T->perm[i] = (int32_t)i;
    }
    if (n == 0) return T;
    int64_t root = new_node(T);
    T->nodes[root].depth = 0;
    T->nodes[root].first = 0;
    T->nodes[root].size = (int)n;
    int32_t *scratch = (int32_t *)malloc(nn * sizeof(int32_t));
    subdivide(T, root, scratch);
    free(scratch);
    return T;
}

/* Batched form: the tree holds one network whose neurons have global ids
 * id_base .. id_base + n - 1; the search draws are keyed by the global id. */
void orc_tree_set_id_base(void *t, int64_t id_base) { ((OTree *)t)->id_base = id_base; }

void orc_tree_free(void *t)
{
    OTree *T = (OTree *)t;
    if (!T) return;
    free(T->px);
    free(T->py);
    free(T->pz);
    free(T->qx);
    free(T->qy);
    free(T->qz);
    free(T->perm);
    free(T->nodes);
    free(T);
}

int64_t orc_tree_num_nodes(void *t) { return ((OTree *)t)->n_nodes; }

void orc_tree_box(void *t, float *lo, float *hi)
{
    OTree *T = (OTree *)t;
    for (int a = 0; a < 3; ++a) {
        lo[a] = T->lo[a];
        hi[a] = T->hi[a];
    }
}

void orc_tree_canonical_order(void *t, int32_t *perm_out)
{
    OTree *T = (OTree *)t;
    memcpy(perm_out, T->perm, (size_t)T->n * sizeof(int32_t));
}

/* ------------------------------------------------------------------------- */
/* Bottom-up update (Sec. III-B "Division of work", first paragraph): a leaf with
 * a neuron has that neuron's vacant dendritic elements and position; an inner
 * node has the sum of its children's counts and their count-weighted average
 * position; a node with no vacant elements has no valid position. */
/* ------------------------------------------------------------------------- */
static void reduce_node(OTree *T, int64_t v, const int32_t *vac_de)
{
    ONode *nv = &T->nodes[v];
    if (nv->leaf) {
        int i = nv->neuron;
        nv->count = (double)vac_de[i];
        nv->sx = nv->count * T->px[i];
        nv->sy = nv->count * T->py[i];
        nv->sz = nv->count * T->pz[i];
    } else {
        double c = 0, sx = 0, sy = 0, sz = 0;
        for (int k = 0; k < nv->nchild; ++k) {
            int64_t ch = nv->child0 + k;
            reduce_node(T, ch, vac_de);
            ONode *nc = &T->nodes[ch];
            c += nc->count;
            sx += nc->sx;
            sy += nc->sy;
            sz += nc->sz;
        }
        nv = &T->nodes[v];
        nv->count = c;
        nv->sx = sx;
        nv->sy = sy;
        nv->sz = sz;
    }
    if (nv->count > 0) {
        nv->cx = nv->sx / nv->count;
        nv->cy = nv->sy / nv->count;
        nv->cz = nv->sz / nv->count;
    } else {
        nv->cx = nv->cy = nv->cz = NAN;
    }
}

void orc_tree_reduce(void *t, const int32_t *vac_de)
{
    OTree *T = (OTree *)t;
    if (T->n_nodes) reduce_node(T, 0, vac_de);
}

/* Export the nodes in pre-order (parent first, children in Morton order).
 * compressed = 1 keeps only the root, leaves and cells with >= 2 children
 * (a cell with a single child cell is the same neuron set as that child). */
static int64_t export_rec(OTree *T, int64_t v, int compressed, int64_t k, int32_t *depth,
                          int32_t *first, int32_t *size, int32_t *is_leaf, int32_t *neuron,
                          double *count, double *cx, double *cy, double *cz)
{
    ONode *nv = &T->nodes[v];
    int keep = !compressed || v == 0 || nv->leaf || nv->nchild >= 2;
    if (keep) {
        if (depth) depth[k] = nv->depth;
        if (first) first[k] = nv->first;
        if (size) size[k] = nv->size;
        if (is_leaf) is_leaf[k] = nv->leaf;
        if (neuron) neuron[k] = nv->leaf ? nv->neuron : -1;
        if (count) count[k] = nv->count;
        if (cx) cx[k] = nv->cx;
        if (cy) cy[k] = nv->cy;
        if (cz) cz[k] = nv->cz;
        ++k;
    }
    for (int c = 0; c < nv->nchild; ++c)
        k = export_rec(T, nv->child0 + c, compressed, k, depth, first, size, is_leaf, neuron,
                       count, cx, cy, cz);
    return k;
}

int64_t orc_tree_export(void *t, int compressed, int32_t *depth, int32_t *first, int32_t *size,
                        int32_t *is_leaf, int32_t *neuron, double *count, double *cx, double *cy,
                        double *cz)
{
    OTree *T = (OTree *)t;
    if (!T->n_nodes) return 0;
    return export_rec(T, 0, compressed, 0, depth, first, size, is_leaf, neuron, count, cx, cy, cz);
}

/* ------------------------------------------------------------------------- */
/* Barnes-Hut partner search (Sec. III-B "Division of work", second paragraph;
 * criterion from Sec. II).
 * Start at the root; the criterion (cell length / distance < theta) rejects the
 * root, and every rejected node is replaced by its children, recursively. One
 * accepted node is drawn with probability proportional to its attraction; a
 * leaf ends the search with a request, an inner node becomes the new start. */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t node;
    double d2;
    double count;
    int self;
} FEntry;

typedef struct {
    FEntry *e;
    int64_t n, cap;
} Frontier;

typedef struct {
    double sigma2, theta2;
    const double *x; /* source position */
    int self;
    /* counters (see orc_search_diag) */
    int64_t evals, expansions, evals_zero;
    double margin_ac;
} SearchCtx;

static void push(Frontier *F, int64_t node, double d2, double count, int self)
{
    if (F->n == F->cap) {
        F->cap = F->cap ? 2 * F->cap : 256;
        F->e = (FEntry *)realloc(F->e, (size_t)F->cap * sizeof(FEntry));
    }
    F->e[F->n].node = node;
    F->e[F->n].d2 = d2;
    F->e[F->n].count = count;
    F->e[F->n].self = self;
    F->n++;
}

/* Expand node v: test each child; accepted ones join the frontier (in child
 * order, which is Morton order, R7), rejected ones are expanded in place.
 * Counters follow the compressed tree: a chain of single-child cells is one
 * node evaluation, so only children of the root or of a branching node count. */
static void expand(const OTree *T, int64_t v, SearchCtx *s, Frontier *F)
{
    const ONode *nv = &T->nodes[v];
    int counted = (v == 0 || nv->nchild >= 2);
    if (counted) s->expansions++;
    for (int k = 0; k < nv->nchild; ++k) {
        int64_t c = nv->child0 + k;
        const ONode *nc = &T->nodes[c];
        if (nc->count == 0) { /* no vacant elements: no valid position */
            if (counted) s->evals_zero++;
            continue;
        }
        if (counted) s->evals++;
        double dx = s->x[0] - nc->cx, dy = s->x[1] - nc->cy, dz = s->x[2] - nc->cz;
        double d2 = dx * dx + dy * dy + dz * dz;
        if (nc->leaf) { /* R4: a single neuron is always accepted */
            push(F, c, d2, nc->count, nc->neuron == s->self);
            continue;
        }
        double len2 = T->len2[nc->depth];
        double rhs = s->theta2 * d2;
        double m = fabs(len2 - rhs) / len2;
        if (m < s->margin_ac) s->margin_ac = m;
        if (len2 < rhs)
            push(F, c, d2, nc->count, 0);
        else
            expand(T, c, s, F);
    }
}

typedef struct {
    int32_t target;      /* neuron id, -1 = failed (R8) */
    int32_t restarts;    /* draws after the first */
    int64_t evals;       /* node evaluations (compressed-tree count, count > 0) */
    int64_t expansions;  /* node expansions (compressed-tree count) */
    int64_t evals_zero;  /* children skipped for count == 0 */
    int64_t frontier0;   /* size of the first (root) frontier */
    double ln_s0;        /* ln of the root frontier's total attraction */
    double margin_ac;    /* min |len^2 - theta^2 d^2| / len^2 over all criterion tests */
    double margin_draw;  /* min |u - C_k / S| over all draws */
} OrcSearchDiag;

/* One search for axonal element e of neuron i. Draws use
 *   u = philox({i, step, (e << 8) | depth(start), 0}, seed).x * 2^-32      (R7)
 * where depth(start) is 0 for the root and the start node's depth after a
 * restart. */
int32_t orc_search(void *t, double sigma, double theta, uint64_t seed, uint64_t step, int32_t i,
                   int32_t e, OrcSearchDiag *diag)
{
    const OTree *T = (const OTree *)t;
    OrcSearchDiag dg;
    memset(&dg, 0, sizeof(dg));
    dg.target = -1;
    dg.margin_ac = INFINITY;
    dg.margin_draw = INFINITY;
    double x[3] = {T->px[i], T->py[i], T->pz[i]};
    SearchCtx s;
    memset(&s, 0, sizeof(s));
    s.sigma2 = sigma * sigma;
    s.theta2 = theta * theta;
    s.x = x;
    s.self = i;
    s.margin_ac = INFINITY;
    Frontier F = {0};
    int64_t start = 0;
    int draws = 0;
    while (T->n_nodes > 0) {
        const ONode *ns = &T->nodes[start];
        F.n = 0;
        if (!ns->leaf) expand(T, start, &s, &F); /* the start node is always expanded */
        if (draws == 0) dg.frontier0 = F.n;
        /* R5 with an exact common factor: shift every exponent by the smallest
         * distance of a candidate that can be drawn, so nothing underflows. */
        double dmin2 = INFINITY;
        for (int64_t k = 0; k < F.n; ++k)
            if (!F.e[k].self && F.e[k].d2 < dmin2) dmin2 = F.e[k].d2;
        double S = 0.0;
        double *a = (double *)malloc((size_t)(F.n ? F.n : 1) * sizeof(double));
        for (int64_t k = 0; k < F.n; ++k) {
            a[k] = F.e[k].self ? 0.0 : F.e[k].count * exp(-(F.e[k].d2 - dmin2) / s.sigma2);
            S += a[k];
        }
        if (draws == 0) dg.ln_s0 = S > 0 ? log(S) - dmin2 / s.sigma2 : -INFINITY;
        if (!(S > 0.0)) { /* R8 */
            free(a);
            break;
        }
        uint32_t w = philox_x((uint32_t)(T->id_base + i), (uint32_t)step,
                              ((uint32_t)e << 8) | (uint32_t)ns->depth, 0u, seed);
        double u = (double)w * (1.0 / 4294967296.0);
        double target = u * S;
        double C = 0.0;
        int64_t pick = -1;
        for (int64_t k = 0; k < F.n; ++k) {
            C += a[k];
            if (k + 1 < F.n) {
                double m = fabs(u - C / S);
                if (m < dg.margin_draw) dg.margin_draw = m;
            }
            if (pick < 0 && target < C) pick = k;
        }
        if (pick < 0) /* u*S rounded up to S: the last candidate with weight */
            for (int64_t k = F.n - 1; k >= 0 && pick < 0; --k)
                if (a[k] > 0) pick = k;
        free(a);
        ++draws;
        int64_t node = F.e[pick].node;
        if (T->nodes[node].leaf) {
            dg.target = T->nodes[node].neuron;
            break;
        }
        start = node; /* restart at the drawn inner node */
    }
    free(F.e);
    dg.restarts = draws > 0 ? draws - 1 : 0;
    dg.evals = s.evals;
    dg.expansions = s.expansions;
    dg.evals_zero = s.evals_zero;
    dg.margin_ac = s.margin_ac;
    if (diag) *diag = dg;
    return dg.target;
}

/* Searches for a list of (neuron, element) queries; optional OpenMP over the
 * independent queries (the tree is read-only here). */
void orc_search_batch(void *t, double sigma, double theta, uint64_t seed, uint64_t step,
                      int64_t nq, const int32_t *qi, const int32_t *qe, int32_t *target,
                      OrcSearchDiag *diag, int threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads > 0 ? threads : 1)
#endif
    for (int64_t q = 0; q < nq; ++q) {
        OrcSearchDiag dg;
        target[q] = orc_search(t, sigma, theta, seed, step, qi[q], qe[q], &dg);
        if (diag) diag[q] = dg;
    }
    (void)threads;
}

int orc_openmp_available(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* Exact distribution of the search outcome from start node v (tiny inputs only):
 * P(j | v) = sum over the frontier of a_k / S * (k leaf ? [k == j] : P(j | k)).
 * Written from the same definitions, used to check the sampler statistically. */
static void marginals_rec(const OTree *T, int64_t v, SearchCtx *s, double w, double *probs)
{
    Frontier F = {0};
    if (!T->nodes[v].leaf) expand(T, v, s, &F);
    double dmin2 = INFINITY;
    for (int64_t k = 0; k < F.n; ++k)
        if (!F.e[k].self && F.e[k].d2 < dmin2) dmin2 = F.e[k].d2;
    double S = 0.0;
    for (int64_t k = 0; k < F.n; ++k)
        if (!F.e[k].self) S += F.e[k].count * exp(-(F.e[k].d2 - dmin2) / s->sigma2);
    if (S > 0.0) {
        for (int64_t k = 0; k < F.n; ++k) {
            if (F.e[k].self) continue;
            double p = w * F.e[k].count * exp(-(F.e[k].d2 - dmin2) / s->sigma2) / S;
            int64_t node = F.e[k].node;
            if (T->nodes[node].leaf)
                probs[T->nodes[node].neuron] += p;
            else
                marginals_rec(T, node, s, p, probs);
        }
    }
    free(F.e);
}

/* probs has n + 1 entries: probs[n] is the failure probability. */
void orc_search_marginals(void *t, double sigma, double theta, int32_t i, double *probs)
{
    const OTree *T = (const OTree *)t;
    memset(probs, 0, (size_t)(T->n + 1) * sizeof(double));
    if (T->n_nodes == 0) return;
    double x[3] = {T->px[i], T->py[i], T->pz[i]};
    SearchCtx s;
    memset(&s, 0, sizeof(s));
    s.sigma2 = sigma * sigma;
    s.theta2 = theta * theta;
    s.x = x;
    s.self = i;
    s.margin_ac = INFINITY;
    marginals_rec(T, 0, &s, 1.0, probs);
    double tot = 0.0;
    for (int64_t j = 0; j < T->n; ++j) tot += probs[j];
    probs[T->n] = 1.0 - tot;
}

/* ------------------------------------------------------------------------- */
/* Acceptance (Sec. III-A "Update of synapses", second sub-phase): each target
 * accepts as many requests as it has vacant dendritic elements, choosing at
 * random (R9); the others are declined and their axonal elements stay vacant. */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t prio;
    int32_t src, elem, idx;
} AKey;

static int cmp_akey(const void *a, const void *b)
{
    const AKey *x = (const AKey *)a, *y = (const AKey *)b;
    if (x->prio != y->prio) return x->prio < y->prio ? -1 : 1;
    if (x->src != y->src) return x->src < y->src ? -1 : 1;
    return (x->elem > y->elem) - (x->elem < y->elem);
}

uint32_t orc_request_priority(uint64_t seed, uint64_t step, int32_t src, int32_t elem)
{
    return philox_x((uint32_t)src, (uint32_t)step, ((uint32_t)elem << 8) | 0xFFu, 1u, seed);
}

/* accept[q] = 1 if request q (src[q], elem[q] -> tgt[q], tgt < 0 = none) is accepted. */
void orc_accept(int64_t n, int64_t nq, const int32_t *src, const int32_t *elem, const int32_t *tgt,
                const int32_t *vac_de, uint64_t seed, uint64_t step, uint8_t *accept)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t q = 0; q < nq; ++q) {
        accept[q] = 0;
        if (tgt[q] >= 0) cnt[tgt[q] + 1]++;
    }
    for (int64_t j = 0; j < n; ++j) cnt[j + 1] += cnt[j];
    AKey *keys = (AKey *)malloc((size_t)(nq ? nq : 1) * sizeof(AKey));
    int64_t *fill = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    for (int64_t j = 0; j < n; ++j) fill[j] = cnt[j];
    for (int64_t q = 0; q < nq; ++q) {
        if (tgt[q] < 0) continue;
        AKey k = {orc_request_priority(seed, step, src[q], elem[q]), src[q], elem[q], (int32_t)q};
        keys[fill[tgt[q]]++] = k;
    }
    for (int64_t j = 0; j < n; ++j) {
        int64_t r = cnt[j + 1] - cnt[j];
        if (r == 0) continue;
        if (r > vac_de[j]) qsort(keys + cnt[j], (size_t)r, sizeof(AKey), cmp_akey);
        int64_t take = r < vac_de[j] ? r : (vac_de[j] > 0 ? vac_de[j] : 0);
        for (int64_t k = 0; k < take; ++k) accept[keys[cnt[j] + k].idx] = 1;
    }
    free(keys);
    free(fill);
    free(cnt);
}

/* ------------------------------------------------------------------------- */
/* Synapse store: the multiset of (src, tgt, sign), kept sorted by (src, tgt)
 * (R12: duplicates counted). */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t src, tgt;
    int8_t sign;
} Syn;

static int cmp_syn(const void *a, const void *b)
{
    const Syn *x = (const Syn *)a, *y = (const Syn *)b;
    if (x->src != y->src) return x->src < y->src ? -1 : 1;
    if (x->tgt != y->tgt) return x->tgt < y->tgt ? -1 : 1;
    return (x->sign > y->sign) - (x->sign < y->sign);
}

/* Apply accepted requests: both ends lose one vacant element and the synapse is
 * added with the source's sign (R10). The store (src, tgt, sign; count *nsyn,
 * capacity cap) is re-sorted into canonical order. Returns the number formed,
 * or -1 if the store would overflow. */
int64_t orc_apply(int64_t nq, const int32_t *src, const int32_t *tgt, const uint8_t *accept,
                  const uint8_t *type, int32_t *vac_ax, int32_t *vac_de, int64_t *nsyn,
                  int64_t cap, int32_t *s_src, int32_t *s_tgt, int8_t *s_sign)
{
    int64_t formed = 0;
    for (int64_t q = 0; q < nq; ++q) formed += accept[q] ? 1 : 0;
    if (*nsyn + formed > cap) return -1;
    int64_t m = *nsyn + formed;
    Syn *all = (Syn *)malloc((size_t)(m ? m : 1) * sizeof(Syn));
    for (int64_t k = 0; k < *nsyn; ++k) {
        all[k].src = s_src[k];
        all[k].tgt = s_tgt[k];
        all[k].sign = s_sign[k];
    }
    int64_t w = *nsyn;
    for (int64_t q = 0; q < nq; ++q) {
        if (!accept[q]) continue;
        vac_ax[src[q]] -= 1;
        vac_de[tgt[q]] -= 1;
        all[w].src = src[q];
        all[w].tgt = tgt[q];
        all[w].sign = type[src[q]] ? -1 : 1;
        ++w;
    }
    qsort(all, (size_t)m, sizeof(Syn), cmp_syn);
    for (int64_t k = 0; k < m; ++k) {
        s_src[k] = all[k].src;
        s_tgt[k] = all[k].tgt;
        s_sign[k] = all[k].sign;
    }
    free(all);
    *nsyn = m;
    return formed;
}

/* ------------------------------------------------------------------------- */
/* Deletion (Sec. III-A "Update of synapses", first sub-phase): a retracted
 * vacant element is simply removed; if all are bound, a random synapse is
 * broken and the partner gains a vacant element (R11).
 * Priorities: axonal side of neuron i, slot k of its out-row (canonical order):
 *   philox({i, step, k, 2}, seed).x; dendritic side of neuron j, slot k of its
 *   in-row (ordered by source, copies in canonical order): philox({j, step, k, 3}).x.
 * Each side breaks the slots with the smallest priorities (ties by slot). */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t prio;
    int32_t slot;
    int64_t syn;
} DKey;

static int cmp_dkey(const void *a, const void *b)
{
    const DKey *x = (const DKey *)a, *y = (const DKey *)b;
    if (x->prio != y->prio) return x->prio < y->prio ? -1 : 1;
    return (x->slot > y->slot) - (x->slot < y->slot);
}

static int cmp_by_tgt_then_pos(const void *a, const void *b)
{
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return (x[1] > y[1]) - (x[1] < y[1]);
}

/* Returns the number of synapses broken. */
int64_t orc_delete(int64_t n, const int32_t *retract_ax, const int32_t *retract_de, int32_t *vac_ax,
                   int32_t *vac_de, uint64_t seed, uint64_t step, int64_t *nsyn, int32_t *s_src,
                   int32_t *s_tgt, int8_t *s_sign)
{
    int64_t m = *nsyn;
    int64_t *need_ax = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *need_de = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *out_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *in_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t k = 0; k < m; ++k) {
        out_ptr[s_src[k] + 1]++;
        in_ptr[s_tgt[k] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) {
        out_ptr[i + 1] += out_ptr[i];
        in_ptr[i + 1] += in_ptr[i];
    }
    /* vacant elements go first */
    for (int64_t i = 0; i < n; ++i) {
        int64_t ra = retract_ax[i] > 0 ? retract_ax[i] : 0;
        int64_t ta = ra < vac_ax[i] ? ra : vac_ax[i];
        vac_ax[i] -= (int32_t)ta;
        ra -= ta;
        int64_t deg = out_ptr[i + 1] - out_ptr[i];
        need_ax[i] = ra < deg ? ra : deg;
        int64_t rd = retract_de[i] > 0 ? retract_de[i] : 0;
        int64_t td = rd < vac_de[i] ? rd : vac_de[i];
        vac_de[i] -= (int32_t)td;
        rd -= td;
        int64_t din = in_ptr[i + 1] - in_ptr[i];
        need_de[i] = rd < din ? rd : din;
    }
    uint8_t *sel_ax = (uint8_t *)calloc((size_t)(m ? m : 1), 1);
    uint8_t *sel_de = (uint8_t *)calloc((size_t)(m ? m : 1), 1);
    DKey *buf = (DKey *)malloc((size_t)(m ? m : 1) * sizeof(DKey));
    /* axonal side: rows of the canonical list */
    for (int64_t i = 0; i < n; ++i) {
        if (!need_ax[i]) continue;
        int64_t b = out_ptr[i], deg = out_ptr[i + 1] - b;
        for (int64_t k = 0; k < deg; ++k) {
            buf[k].prio = philox_x((uint32_t)i, (uint32_t)step, (uint32_t)k, 2u, seed);
            buf[k].slot = (int32_t)k;
            buf[k].syn = b + k;
        }
        qsort(buf, (size_t)deg, sizeof(DKey), cmp_dkey);
        for (int64_t k = 0; k < need_ax[i]; ++k) sel_ax[buf[k].syn] = 1;
    }
    /* dendritic side: in-rows = canonical list stably ordered by target */
    int64_t *order = (int64_t *)malloc((size_t)(m ? m : 1) * 2 * sizeof(int64_t));
    for (int64_t k = 0; k < m; ++k) {
        order[2 * k] = s_tgt[k];
        order[2 * k + 1] = k;
    }
    qsort(order, (size_t)m, 2 * sizeof(int64_t), cmp_by_tgt_then_pos);
    for (int64_t j = 0; j < n; ++j) {
        if (!need_de[j]) continue;
        int64_t b = in_ptr[j], deg = in_ptr[j + 1] - b;
        for (int64_t k = 0; k < deg; ++k) {
            buf[k].prio = philox_x((uint32_t)j, (uint32_t)step, (uint32_t)k, 3u, seed);
            buf[k].slot = (int32_t)k;
            buf[k].syn = order[2 * (b + k) + 1];
        }
        qsort(buf, (size_t)deg, sizeof(DKey), cmp_dkey);
        for (int64_t k = 0; k < need_de[j]; ++k) sel_de[buf[k].syn] = 1;
    }
    int64_t w = 0, broken = 0;
    for (int64_t k = 0; k < m; ++k) {
        if (sel_ax[k] || sel_de[k]) {
            ++broken;
            if (sel_ax[k] && !sel_de[k]) vac_de[s_tgt[k]] += 1;
            if (sel_de[k] && !sel_ax[k]) vac_ax[s_src[k]] += 1;
            continue;
        }
        s_src[w] = s_src[k];
        s_tgt[w] = s_tgt[k];
        s_sign[w] = s_sign[k];
        ++w;
    }
    *nsyn = w;
    free(order);
    free(buf);
    free(sel_ax);
    free(sel_de);
    free(need_ax);
    free(need_de);
    free(out_ptr);
    free(in_ptr);
    return broken;
}

/* ------------------------------------------------------------------------- */
/* Spike delivery (Sec. III-A "Update of electrical activity"): spikes travel
 * over synapses; the input of t is the signed sum over its incoming synapses
 * of the sources that spiked (duplicates count). */
/* ------------------------------------------------------------------------- */
void orc_deliver_spikes(int64_t n, int64_t nsyn, const int32_t *s_src, const int32_t *s_tgt,
                        const int8_t *s_sign, const uint8_t *spiked, int32_t *input)
{
    for (int64_t t = 0; t < n; ++t) input[t] = 0;
    for (int64_t k = 0; k < nsyn; ++k)
        if (spiked[s_src[k]]) input[s_tgt[k]] += s_sign[k];
}

/* ------------------------------------------------------------------------- */
/* Firing-rate delivery (Sec. IV-B "Approximation of firing rates"): instead of
 * receiving spikes, a neuron uses the sender's firing frequency and a PRNG to
 * decide whether the sender spiked in this step (R13). */
/* ------------------------------------------------------------------------- */
void orc_deliver_rates(int64_t n, int64_t nsyn, const int32_t *s_src, const int32_t *s_tgt,
                       const int8_t *s_sign, const float *rate, uint64_t seed, uint64_t step,
                       int32_t *input)
{
    for (int64_t t = 0; t < n; ++t) input[t] = 0;
    for (int64_t k = 0; k < nsyn; ++k) {
        uint32_t w = philox_x((uint32_t)s_src[k], (uint32_t)s_tgt[k], (uint32_t)step, 4u, seed);
        if ((double)w < (double)rate[s_src[k]] * 4294967296.0) input[s_tgt[k]] += s_sign[k];
    }
}

/* ------------------------------------------------------------------------- */
/* Differentiable form (not in the paper; reading R15). The expected synapse
 * length of a source i over its root frontier F_i -- the candidates of its first
 * draw (Sec. III-B, criterion of Sec. II), own leaf excluded (R6):
 *   D_ik = |x_i - c_k|^2, d_ik = sqrt(D_ik), a_ik = N_k exp(-D_ik / sigma^2) (R5),
 *   S_i = sum_k a_ik, q_ik = a_ik / S_i, l_i = sum_k q_ik d_ik,
 *   L = sum_i m_i l_i / M, M = sum_i m_i over the sources with m_i > 0, S_i > 0
 * (m = vac_ax: the searches a source makes). Gradients; the criterion and the
 * tree topology are piecewise constant and contribute nothing:
 *   dl_i/dsigma = (2 / sigma^3) sum_k q_ik (d_ik - l_i) (D_ik - Dbar_i),
 *                 Dbar_i = sum_k q_ik D_ik,
 *   dl_i/dc_k   = q_ik r_ik (2 (d_ik - l_i) / sigma^2 - 1 / d_ik), r = x_i - c_k
 *                 (the 1/d term is 0 where d = 0),
 *   dl_i/dx_i   = -sum_k dl_i/dc_k,
 *   dc_k/dx_j   = w_j / N_k for every neuron j in cell k (w = vac_de: the
 *                 bottom-up centroid is the w-weighted mean).
 * ell (per neuron, NAN for excluded sources), dsigma and the position
 * gradients gx, gy, gz are optional outputs; returns L (NAN when M = 0).
 * margin (optional, per neuron) is a diagnostic for the comparison with FP32:
 * min |len^2 - theta^2 d^2| / len^2 over the criterion tests of the source's
 * root frontier (INFINITY when there are none or the neuron is no source).
 * ax, ay, az (optional, with the gradients) are the same sums as gx, gy, gz taken
 * over the magnitudes of their terms: the scale against which the rounding error of
 * a sum of terms of both signs is measured (|g| <= a, equal without cancellation).
 * Optional OpenMP over the independent sources (threads). */
/* ------------------------------------------------------------------------- */
static int root_frontier(const OTree *T, int32_t i, double sigma, double theta, Frontier *F,
                         double *a, double *S_out, double *margin_out)
{
    double x[3] = {T->px[i], T->py[i], T->pz[i]};
    SearchCtx s;
    memset(&s, 0, sizeof(s));
    s.sigma2 = sigma * sigma;
    s.theta2 = theta * theta;
    s.x = x;
    s.self = i;
    s.margin_ac = INFINITY;
    F->n = 0;
    if (margin_out) *margin_out = INFINITY;
    if (T->n_nodes == 0 || T->nodes[0].leaf) {
        *S_out = 0.0;
        return 0;
    }
    expand(T, 0, &s, F);
    if (margin_out) *margin_out = s.margin_ac;
    double dmin2 = INFINITY; /* common factor exp(dmin2 / sigma^2): q is unchanged */
    for (int64_t k = 0; k < F->n; ++k)
        if (!F->e[k].self && F->e[k].d2 < dmin2) dmin2 = F->e[k].d2;
    double S = 0.0;
    for (int64_t k = 0; k < F->n; ++k) {
        a[k] = F->e[k].self ? 0.0 : F->e[k].count * exp(-(F->e[k].d2 - dmin2) / s.sigma2);
        S += a[k];
    }
    *S_out = S;
    return 1;
}

double orc_mean_length(void *t, double sigma, double theta, const int32_t *vac_ax,
                       const int32_t *vac_de, double *ell, double *dsigma, double *gx,
                       double *gy, double *gz, double *margin, double *ax, double *ay,
                       double *az, int threads)
{
    const OTree *T = (const OTree *)t;
    const int64_t n = T->n;
    double *lsrc = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
    double M = 0.0, sum = 0.0, sdsig = 0.0;
    if (threads < 1) threads = 1;
    /* pass 1: l_i and dl_i/dsigma (sources are independent) */
#ifdef _OPENMP
#pragma omp parallel num_threads(threads) reduction(+ : M, sum, sdsig)
#endif
    {
        double *a = (double *)malloc((size_t)(n + 1) * sizeof(double));
        Frontier F = {0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t i = 0; i < n; ++i) {
            lsrc[i] = NAN;
            if (margin) margin[i] = INFINITY;
            if (vac_ax[i] <= 0) continue;
            double S;
            root_frontier(T, (int32_t)i, sigma, theta, &F, a, &S, margin ? &margin[i] : NULL);
            if (!(S > 0.0)) continue;
            double l = 0.0, Db = 0.0;
            for (int64_t k = 0; k < F.n; ++k) {
                double q = a[k] / S;
                l += q * sqrt(F.e[k].d2);
                Db += q * F.e[k].d2;
            }
            double cov = 0.0;
            for (int64_t k = 0; k < F.n; ++k)
                cov += a[k] / S * (sqrt(F.e[k].d2) - l) * (F.e[k].d2 - Db);
            lsrc[i] = l;
            M += vac_ax[i];
            sum += vac_ax[i] * l;
            sdsig += vac_ax[i] * 2.0 / (sigma * sigma * sigma) * cov;
        }
        free(F.e);
        free(a);
    }
    if (ell) memcpy(ell, lsrc, (size_t)n * sizeof(double));
    if (dsigma) *dsigma = M > 0 ? sdsig / M : NAN;
    if (gx && gy && gz) {
        /* pass 2: dL/dc_k accumulated per node (G), direct terms per source */
        double *G = (double *)calloc((size_t)(T->n_nodes ? T->n_nodes : 1) * 3, sizeof(double));
        const int mag = ax && ay && az;
        double *Ga = mag ? (double *)calloc((size_t)(T->n_nodes ? T->n_nodes : 1) * 3,
                                            sizeof(double))
                         : NULL;
        for (int64_t j = 0; j < n; ++j) gx[j] = gy[j] = gz[j] = 0.0;
        if (mag)
            for (int64_t j = 0; j < n; ++j) ax[j] = ay[j] = az[j] = 0.0;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
#endif
        {
            double *a = (double *)malloc((size_t)(n + 1) * sizeof(double));
            Frontier F = {0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int64_t i = 0; i < n; ++i) {
                if (!(M > 0) || !(lsrc[i] == lsrc[i])) continue; /* excluded source */
                double S;
                root_frontier(T, (int32_t)i, sigma, theta, &F, a, &S, NULL);
                const double w = vac_ax[i] / M, l = lsrc[i];
                for (int64_t k = 0; k < F.n; ++k) {
                    if (F.e[k].self || a[k] == 0.0) continue;
                    const ONode *nk = &T->nodes[F.e[k].node];
                    double r[3] = {T->px[i] - nk->cx, T->py[i] - nk->cy, T->pz[i] - nk->cz};
                    double d = sqrt(F.e[k].d2);
                    double kap =
                        a[k] / S * (2.0 * (d - l) / (sigma * sigma) - (d > 0 ? 1.0 / d : 0.0));
                    for (int c = 0; c < 3; ++c) {
                        double g = w * kap * r[c];
#ifdef _OPENMP
#pragma omp atomic
#endif
                        G[3 * F.e[k].node + c] += g;
                        (c == 0 ? gx : c == 1 ? gy : gz)[i] -= g;
                        if (mag) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                            Ga[3 * F.e[k].node + c] += fabs(g);
                            (c == 0 ? ax : c == 1 ? ay : az)[i] += fabs(g);
                        }
                    }
                }
            }
            free(F.e);
            free(a);
        }
        /* scatter: neuron j gets w_j * sum over the cells that hold it of G_k / N_k */
        for (int64_t v = 0; v < T->n_nodes; ++v) {
            const ONode *nv = &T->nodes[v];
            if (!nv->leaf) continue;
            int j = nv->neuron;
            double h[3] = {0, 0, 0}, ha[3] = {0, 0, 0};
            for (int64_t u = v; u >= 0; u = T->nodes[u].parent) {
                const ONode *nu = &T->nodes[u];
                if (nu->count > 0)
                    for (int c = 0; c < 3; ++c) {
                        h[c] += G[3 * u + c] / nu->count;
                        if (mag) ha[c] += Ga[3 * u + c] / nu->count;
                    }
            }
            gx[j] += vac_de[j] * h[0];
            gy[j] += vac_de[j] * h[1];
            gz[j] += vac_de[j] * h[2];
            if (mag) {
                ax[j] += vac_de[j] * ha[0];
                ay[j] += vac_de[j] * ha[1];
                az[j] += vac_de[j] * ha[2];
            }
        }
        free(G);
        free(Ga);
    }
    free(lsrc);
    return M > 0 ? sum / M : NAN;
}
