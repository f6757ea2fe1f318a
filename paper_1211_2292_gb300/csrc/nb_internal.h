// Internal declarations shared by the CUDA translation units and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "nbody.h"

namespace nb {

// Error-word bits (ctx scratch, read by nb_sync / nb_energy): a non-finite
// result; a tree that outgrew its node arrays.
enum : int { ERR_NONFINITE = 1, ERR_TREE = 2 };
// Kernel families with autotuned variants (the `kind` of nb_variant_*).
enum Kind : int { KIND_FORCE = 0, KIND_BATCHED = 1, KIND_VJP = 2, KIND_COUNT = 3 };
// Event-timing tags of nb_profile_read: 0-2 the kinds above, then these.
enum ProfKind : int { PROF_ENERGY = 3, PROF_TREE_WALK = 4, PROF_TREE_BUILD = 5, PROF_FMM_FAR = 6,
                      PROF_FMM_NEAR = 7 };

// One compiled kernel: CTA shape plus the function to launch.  Every kernel
// of a family takes a single by-value parameter struct.
struct KernelEntry {
    int T;   // threads per CTA
    int I;   // i-bodies per thread
    int J;   // j-bodies per shared-memory tile
    const void *fn;
    bool logm = false;  // float32 kernels with log-domain pairs (read log2 m from P_lo.w)
};

// -------------------------------------------------------------- parameters
struct ForceParams {
    const void *P;        // packed bodies: float4 (x_hi,y_hi,z_hi,m) or double4 (x,y,z,m)
    const float4 *Plo;    // float32 modes: (x_lo,y_lo,z_lo,0), x = x_hi + x_lo
    const int *perm;      // float32 modes: body stored at packed slot k (NULL = identity)
    int n;                // bodies
    int nsplit;           // j-splits across CTAs (grid = i-tiles * nsplit)
    float eps2f;          // eps^2 in float32
    double eps2;          // eps^2 in float64
    double G;
    double *acc;          // out [n][3]
    double *vel;          // optional fused half-kick: vel += half_dt * acc
    double half_dt;
    double *partial;      // [nsplit][n][3] split partial sums (nsplit > 1)
    unsigned *counters;   // per-i-tile arrival counters, zero between launches
    int *err;             // error word
};

// One work item of the batched kernel: bodies [i0, i_end) of one system,
// interacting with bodies [j0, j1) of the same system, `lanes` adjacent
// threads splitting the j loop of each body (the CTA then covers
// threads * bodies_per_thread / lanes bodies).  A piece of a system whose
// j range is split over nchunks > 1 items ("chunks", j-tile aligned) has
// arrival counter `ctr`; chunk c stores its float64 partial sums in partial
// slot pbase + c, and the last chunk to arrive adds the slots in chunk order.
// nchunks == 1: ctr = -1, the item writes its bodies' accelerations itself.
struct BatchItem {
    int i0, i_end, j0, j1;
    int lanes, sys, ctr, pbase;
    int chunk, nchunks, pad0, pad1;
};
constexpr int BATCH_ITEM_INTS = 12;

struct BatchParams {
    const float4 *P;      // (x_hi,y_hi,z_hi,m)
    const float4 *Plo;    // (x_lo,y_lo,z_lo,0)
    const BatchItem *items;
    int n_items;
    unsigned *queue;      // [0] next item, [1] CTAs done; both zero between launches
    double *partial;      // [slots][threads * bodies_per_thread][3] chunk partial sums
    unsigned *counters;   // per split piece, zero between launches
    float eps2f;
    double G;
    double *acc;
    double *vel;
    double half_dt;
    int *err;
};

struct VjpParams {
    const void *PV;       // float64: (x,y,z,m),(mu_x,mu_y,mu_z,0) per body (double4 pairs);
                          // float32: (x_hi,y_hi,z_hi,m) per body
    const float4 *Plo;    // float32: (x_lo,y_lo,z_lo,.)
    const float4 *Plam;   // float32: (mu_x,mu_y,mu_z,0)
    int n;
    int nsplit;
    float eps2f;
    double eps2;
    double G;
    double *gx;           // [n][3]
    double *gm;           // [n]
    int accumulate;       // 0: overwrite gx/gm with G*sum; 1: add G*sum
    double *partial;      // [nsplit][n][4]
    unsigned *counters;
    int *err;
};

struct EnergyParams {
    const double4 *P;     // packed float64 bodies
    const double *vel;    // [n][3]
    int n;
    int nsplit;
    double eps2;
    double *red;          // [grid][8] per-CTA partial sums
    int *err;
};

// ----------------------------------------------------------- kernel tables
// Defined in force_f32*.cu / force_f64.cu / adjoint.cu.  Index [variant][comp][zero_eps].
int f32_force_variants_a();
const KernelEntry &f32_force_kernel_a(int variant, bool comp, bool zeps);
int f32_force_variants_b();
const KernelEntry &f32_force_kernel_b(int variant, bool comp, bool zeps);
int f32_force_variants();
const KernelEntry &f32_force_kernel(int variant, bool comp, bool zeps);
int f32_batched_variants();
const KernelEntry &f32_batched_kernel(int variant, bool comp, bool zeps);
int f64_force_variants();
const KernelEntry &f64_force_kernel(int variant, bool zeps);
int df_force_variants();  // double-float (float32-pipe, float64-accurate) force kernels
const KernelEntry &df_force_kernel(int variant, bool zeps);
const KernelEntry &f64_energy_kernel(bool zeps);
int f32_vjp_variants();
const KernelEntry &f32_vjp_kernel(int variant, bool zeps);
int f64_vjp_variants();
const KernelEntry &f64_vjp_kernel(int variant, bool zeps);

// -------------------------------------------------- spatial order (order.cu)
constexpr int SORT_CHUNK = 2048;  // keys per warp-chunk of the radix sort
struct OrderScratch {
    double *box;        // [1024][6]: bounding-box partials of up to 1023 blocks, then the folded box
    unsigned *keys[2];  // [n] Morton keys (ping-pong)
    int *vals[2];       // [n] body indices (ping-pong)
    unsigned *hist;     // [256][chunks] digit counts / offsets, then scan partials
};
int sort_chunks(int n);
size_t sort_hist_entries(int n);  // entries of OrderScratch::hist for n bodies
// perm_out[k] = body at Morton rank k (stable in body index); `kernels` = launches made.
cudaError_t launch_morton_sort(cudaStream_t s, int n, const double *pos, OrderScratch &o,
                               int *perm_out, int &kernels);
// Tree-code order: 30-bit Morton keys (float64 quantisation), stable radix
// sort; sorted keys end in o.keys[0], box_out = {lo_x, lo_y, lo_z, ext}.
cudaError_t launch_tree_sort(cudaStream_t s, int n, const double *pos, OrderScratch &o,
                             int *perm_out, double *box_out, int &kernels);
// Stable sort of bodies by an integer key below 2^(8 passes) (k32, or k64
// when k32 is NULL; values below 2^31): perm_out[k] = the k-th body.
cudaError_t launch_key_sort(cudaStream_t s, int n, const int *k32, const long long *k64,
                            int passes, OrderScratch &o, int *perm_out, int &kernels);
// Phi[k], Plo[k] = float32 hi/lo packing of body perm[k] (perm NULL = identity);
// Phi.w = m, Plo.w = log2(m).
cudaError_t launch_pack_hilo(cudaStream_t s, int n, const double *pos, const double *mass,
                             const int *perm, float4 *Phi, float4 *Plo);

// ------------------------------------------------------ tree code (tree.cu)
// Octree over bodies in 30-bit Morton order.  Node arrays hold `cap` entries;
// a node covers sorted bodies [start, end), sits at `level` with key prefix
// `prefix` (3 * level bits), and has `nchild` children stored contiguously
// from `first` in octant order (nchild == 0: leaf).
struct TreeView {
    int cap;
    int *meta;            // [tree_meta_ints()] per-level node counts and bases, overflow flag
    int *start, *end, *level, *nchild, *first, *offs;
    int *parent, *arrive;     // parent node (-1 at the root); children counted in by the moments
    unsigned *prefix;
    double *M, *com;      // float64 monopoles: mass, centre of mass [cap][3]
    float4 *box_lo, *box_hi;  // float32 cell cube corners; .w = nchild, first (int bits)
    float4 *chi, *clo;    // centre of mass hi/lo float32 pair; chi.w = mass
    unsigned long long *stats;  // [4] nodes, leaves, cell and body interactions
};
// A further tree walked after TreeWalkParams::tree in the same launch (a
// received LET): its walk data, the bodies its leaves index, its cube.
struct WalkSource {
    const float4 *box_lo, *box_hi, *chi, *clo;
    const int *start, *end;
    const float4 *sP, *sPlo;
    const double *box;
};
constexpr int WALK_MAX_MORE = 63;  // further trees per launch

struct TreeWalkParams {
    TreeView tree;          // the tree walked (the targets' own, or a received LET)
    const float4 *P, *Plo;  // target bodies in their own tree's order, float32 hi/lo
    const int *perm;        // target tree rank -> body index
    const float4 *sP, *sPlo;  // source bodies the walked tree's leaves index
    const double *box;      // walked tree's cube {lo_x, lo_y, lo_z, ext}
    int *queue;             // group queue of the dynamic schedules, zero at launch
    int n;
    int group;              // bodies per walking warp: 32 or 64
    int sched, chunk;       // group schedule: 0 static, 1 dynamic, 2 guided; chunk size
    int num_sms;
    int accumulate;         // 1: add to acc and counts (vel must be NULL)
    float theta, eps2f;
    double G;
    double *acc, *vel;      // vel != NULL: vel += half_dt * acc
    double half_dt;
    int *counts;            // optional [n][2]: cells, bodies met per body
    int *err;
    const WalkSource *more;  // device [1 + nmore] when nmore > 0: `tree` (again) and the trees
    int nmore;               // walked after it, their sums added in order (as separate
                             // accumulating walks would); nmore 0..WALK_MAX_MORE
    // Split mode (nmore > 0): one task per group and span of tspan trees; each
    // writes its span's sums, the group's last task adds them in tree order.
    int tspan;               // trees per task (1: every tree's sum added in turn)
    double *tpart;           // [spans][groups * group][3] per-span sums, group order
    int *tcnt;               // [spans][groups][2] per-span cells, bodies met
    unsigned *tctr;          // [groups] tasks arrived; zero between launches
};
int tree_meta_ints();
// Upper bound on the node count of a tree over n bodies with leaves of at
// most leaf_cap bodies (no build can exceed it).
int64_t tree_node_bound(int64_t n, int leaf_cap);
// Build over sorted keys (launch_tree_sort), float64 moments, float32 walk data.
// box = {lo_x, lo_y, lo_z, ext} from launch_tree_sort.
cudaError_t launch_tree_build(cudaStream_t s, const TreeView &t, int n, const unsigned *keys,
                              const double *box, const double *pos, const double *mass,
                              const int *perm, int leaf_cap, int *err, int &kernels);
cudaError_t launch_tree_walk(cudaStream_t s, const TreeWalkParams &p, bool zeps, int &kernels);
// Where tree.cu keeps each level's node count and first node, and the walk's
// group queue, in TreeView::meta.
constexpr int TREE_META_COUNT = 0, TREE_META_BASE = 12, TREE_META_QUEUE = 25;

// ------------------------------------ locally essential trees (tree.cu)
// A LET is one contiguous device buffer: a header, then per node the cube
// corners (.w: child count, first child, as in TreeView), the centre of mass
// hi/lo pair, the leaf's body range, then the bodies (float32 hi/lo).  Node
// order is the source tree's (level by level, children of a node
// consecutive); levels are the source's, so the walk's opening distances
// come from the header's box.
struct LetHeader {
    long long magic, n_nodes, n_bodies, reserved;
    double box[4];  // the source tree's {lo_x, lo_y, lo_z, ext}
};
constexpr long long LET_MAGIC = 0x31305445'4c424e;  // identifies a LET buffer
struct LetLayout {
    size_t lo, hi, chi, clo, start, end, P, Plo, total;  // byte offsets; total size
};
__host__ __device__ inline size_t let_round16(size_t b) { return (b + 15) & ~(size_t)15; }
__host__ __device__ inline LetLayout let_layout(long long nn, long long nb)
{
    LetLayout L;
    L.lo = sizeof(LetHeader);
    L.hi = L.lo + 16 * (size_t)nn;
    L.chi = L.hi + 16 * (size_t)nn;
    L.clo = L.chi + 16 * (size_t)nn;
    L.start = L.clo + 16 * (size_t)nn;
    L.end = L.start + let_round16(4 * (size_t)nn);
    L.P = L.end + let_round16(4 * (size_t)nn);
    L.Plo = L.P + 16 * (size_t)nb;
    L.total = L.Plo + 16 * (size_t)nb;
    return L;
}
// Per-node scratch of the LET selection: kind (0 not sent, 1 sent alone,
// 2 sent with its children, 3 a leaf sent with its bodies), the node's
// index in the LET and its first body there; totals = {nodes, bodies}.
struct LetScratch {
    int *kind, *nidx, *boff, *totals;
};
// Kinds and LET indices of the nodes of tree t (built over the bodies whose
// packed float32 pairs the leaves index) for a destination whose bodies lie
// in the float32 box [dlo, dhi]; then totals holds {nodes, bodies}.
cudaError_t launch_let_select(cudaStream_t s, const TreeView &t, const double *box, float theta,
                              float3 dlo, float3 dhi, const LetScratch &sc, int &kernels);
// Writes the LET selected by launch_let_select into out (let_layout(totals) bytes).
cudaError_t launch_let_emit(cudaStream_t s, const TreeView &t, const double *box,
                            const LetScratch &sc, const float4 *P, const float4 *Plo, void *out,
                            int &kernels);

// ------------------------------------------------- fast multipole method (fmm.cu)
// Expansion orders with compiled kernels, and floats per expansion (the
// (p+1)(p+2)(p+3)/6 coefficients padded to a multiple of 4).
constexpr int FMM_MIN_ORDER = 2, FMM_MAX_ORDER = 6, FMM_MAX_LEAF = 64;
int fmm_floats(int order);
enum : int { FMM_META_LEVEL = 0, FMM_META_NEAR = 11, FMM_META_POOL = 12, FMM_META_OVERFLOW = 13,
             FMM_META_NLEAVES = 14, FMM_META_ITEMS = 15, FMM_META_PSLOTS = 16,
             FMM_META_CHUNKS = 17, FMM_META_M2L = 18, FMM_META_LEAVES_Q = 19, FMM_META_RCHUNKS = 20,
             FMM_META_INTS = 24 };
// FMM_META_OVERFLOW bits: the candidate pool (1), the expansion-list chunks
// (2), the direct-range chunks (4).
constexpr int FMM_CHUNK = 32;  // source ids per expansion-list chunk
constexpr int FMM_CRIT_INTS = 2 * 11 * 11;  // two thresholds per pair of tree levels
struct FmmView {
    int order, np;         // expansion order p; floats per expansion
    int4 *ci;              // per node: integer centre in units ext/2048 (.xyz), level (.w)
    int4 *nd;              // per node: child count, first child, first body, end of bodies
    float *M, *L;          // [cap][np]: scaled moments, scaled local coefficients
    int2 *down;            // per node: (offset, count) in pool of the candidates handed to its children
    int2 *cum;             // per node: source cells acting on it and its ancestors, bodies they hold
    int *leaves;           // leaf ids, in the order the downward pass meets them
    int *nearc;            // per node (leaves): bodies met directly
    int *item_off;         // per leaf index: first near-field work item (exclusive scan)
    int *part_off;         // per leaf index: first partial-sum slot (leaves split in several items)
    double *part;          // [slots][3] partial direct sums of split leaves
    long long part_cap;    // slots part holds
    int *pool;             // candidate lists; pool[0] = 0, the root's own list
    long long pool_cap;
    int *chunk_head;       // per node: its expansion list's first chunk, -1 for none
    int *chunk_src;        // [chunk_cap][FMM_CHUNK] source cells, -1 past a list's end
    int *chunk_next;       // [chunk_cap] the next chunk of the same list, -1 at the end
    long long chunk_cap;
    int *rhead;            // per leaf: first chunk of its directly summed cells, -1 for none
    int2 *rchunk;          // [rchunk_cap][FMM_CHUNK] those cells' body ranges, (0, 0) past the end
    int *rnext;            // [rchunk_cap] the next chunk of the same list, -1 at the end
    long long rchunk_cap;
    int *meta;             // [FMM_META_INTS] queues, pool top, overflow flag, leaf count
    int *crit;             // [FMM_CRIT_INTS] the cell tests' thresholds for this evaluation's theta
    unsigned long long *stats;  // [4] nodes, leaves, expansions, direct body pairs
};
struct FmmParams {
    TreeView tree;
    FmmView f;
    const float4 *P, *Plo;  // bodies in tree order, float32 hi/lo
    const int *perm;        // tree rank -> body index
    const double *pos, *mass;
    const double *box;      // {lo_x, lo_y, lo_z, ext}
    int n;
    double theta, eps2;
    float eps2f;
    double G;
    double *acc;
    double *vel;            // vel != NULL: vel += half_dt * acc
    double half_dt;
    int *counts;            // optional [n][3]
    int *err;
    int num_sms;
};
// near = false: upward pass, downward levels, near-field work items (the
// host then reads the meta counters); near = true: the near field.
cudaError_t launch_fmm(cudaStream_t s, const FmmParams &p, bool near, int &kernels);

// ------------------------------------ orthogonal recursive bisection (orb.cu)
// Group ids are the first processor of a part; `slot` maps a group id to
// its row in the per-part tables (-1: the part is not being cut).
constexpr int ORB_MAX_P = NB_ORB_MAX_P;
struct OrbTables {
    int slot[ORB_MAX_P];                 // group id -> active row
    int axis[ORB_MAX_P / 2];             // per active row: the cut axis
    int upper[ORB_MAX_P / 2];            // per active row: group id of the upper part
    unsigned long long key_hi[ORB_MAX_P / 2];  // prefix (hist) or split key (cut), high 64 bits
    unsigned key_lo[ORB_MAX_P / 2];      // low 32 bits (the body id)
};
// box[g][6] (order-preserving images: min xyz, max xyz) of each group's bodies.
cudaError_t launch_orb_box(cudaStream_t s, int n, const double *pos, const int *group, int ngroups,
                           unsigned long long *box);
// hist[row][256]: digit `round` (0..11, most significant first) of the
// 96-bit key (coordinate image, body id) of the bodies whose key starts
// with the row's prefix.
cudaError_t launch_orb_hist(cudaStream_t s, int n, const double *pos, const long long *id,
                            const int *group, int nactive, const OrbTables &t, int round,
                            unsigned long long *hist);
// Bodies of an active part with key >= the row's split key move to `upper`.
cudaError_t launch_orb_cut(cudaStream_t s, int n, const double *pos, const long long *id,
                           int *group, const OrbTables &t);
// out[k] = body perm[k] (any output may be NULL); counts[r] = bodies with rank r.
cudaError_t launch_gather_bodies(cudaStream_t s, int n, const int *perm, const double *pos,
                                 const double *vel, const double *mass, const long long *id,
                                 double *pos_out, double *vel_out, double *mass_out,
                                 long long *id_out);
cudaError_t launch_rank_counts(cudaStream_t s, int n, const int *rank, int P,
                               unsigned long long *counts);
// Float32 bounding box {min xyz, max xyz} of n packed bodies (their hi parts).
cudaError_t launch_hi_box(cudaStream_t s, int n, const float4 *P, float *box);

// ------------------------------------------------- O(n) kernels (integrate.cu)
cudaError_t launch_pack_f32(cudaStream_t s, int n, const double *pos, const double *mass, float4 *P);
// P[k] = (x, y, z, m) of body perm[k] (perm NULL = identity).
cudaError_t launch_pack_f64(cudaStream_t s, int n, const double *pos, const double *mass, double4 *P,
                            const int *perm = nullptr);
// v += half_dt a; x += dt v; then repack into P (double4) when f64, into the
// float32 hi/lo pair (P, Plo) otherwise; P == NULL skips the packing.  Records
// (x, v) before the update when rec_* is set.
cudaError_t launch_kdp(cudaStream_t s, bool f64, int n, double *pos, double *vel, const double *acc,
                       const double *mass, double half_dt, double dt, void *P, float4 *Plo,
                       double *rec_pos, double *rec_vel);
// Adjoint packing: lam_v += drift * lam_x (if lam_x), mu = coef * lam_v, pack (x, m, mu):
// float64 as double4 pairs at PV[2i], PV[2i+1]; float32 as three float4 arrays
// PV[i] = (x_hi,y_hi,z_hi,m), PV[stride + i] = (x_lo,..,0), PV[2 stride + i] = (mu,0).
cudaError_t launch_pack_vjp(cudaStream_t s, bool f64, int n, const double *pos, const double *mass,
                            const double *lam, double *lam_v, const double *lam_x, double drift,
                            double coef, void *PV, size_t stride);
cudaError_t launch_energy_final(cudaStream_t s, const double *red, int nparts, double G, double *out);

// Host-side scheduling helpers (nbody_abi.cpp; exported for tests).
int choose_split(int64_t n_itiles, int64_t n_jtiles, int64_t slots, int64_t max_split_bodies,
                 int64_t tile_bodies);

}  // namespace nb

// ------------------------------------------------------------------ context
struct nb_ctx {
    int device = 0;
    int num_sms = 0;
    nb_precision prec = NB_FP64;
    int64_t n_max = 0;
    cudaStream_t stream = nullptr;      // caller's stream
    cudaStream_t cap_stream = nullptr;  // library stream used for graph capture/launch
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;

    // scratch
    void *pack = nullptr;        // packed bodies (force/energy/VJP)
    size_t pack_bytes = 0;
    double *partial = nullptr;   // split partials
    int64_t partial_bodies = 0;  // capacity in body-splits (4 doubles each)
    unsigned *counters = nullptr;
    int64_t n_counters = 0;
    double *red = nullptr;       // energy per-CTA partials
    int64_t n_red = 0;           // capacity in CTAs
    int *perm = nullptr;         // spatial order of the last float32 force call
    bool perm_active = false;    // the packed bodies are in perm order
    nb::OrderScratch order{};
    int order_mode = 2;          // 0 never, 1 always, 2 when n >= order_min_n
    int64_t order_min_n = 131072;
    double *dev_out = nullptr;   // 16 doubles
    double *host_out = nullptr;  // pinned, 16 doubles
    int *err = nullptr;
    unsigned *queue = nullptr;   // batched queue counters [2]

    // batched plan
    nb::BatchItem *items = nullptr;
    int64_t n_items = 0, items_cap = 0;
    int batch_variant = 0;
    int64_t batch_n = 0;         // bodies covered by the plan
    int64_t batch_nsys = 0;
    uint64_t plan_gen = 0;

    // tuning: per kind, list of (lo, hi, variant, split)
    struct TuneEntry { int64_t lo, hi; int variant, split; };
    std::vector<TuneEntry> tune[nb::KIND_COUNT];

    // graph cache for nb_step_batched
    struct GraphKey {
        int kind;  // 0: nb_rollout, 1: nb_step_batched
        const void *pos, *vel, *mass, *acc, *rec_pos, *rec_vel;
        double G, eps, dt;
        int64_t n, nsteps, every;
        unsigned flags;
        uint64_t plan_gen;
        double theta = 0.0;  // tree code only
        int leaf_cap = 0;    // tree code only: leaf_cap * 128 + group
        bool operator<(const GraphKey &o) const;
    };
    struct GraphVal { cudaGraphExec_t exec; int64_t kernels; };
    std::map<GraphKey, GraphVal> graphs;

    // tree code scratch (allocated on first use; bodies sized for n_max)
    nb::TreeView tree{};
    int tree_sched = 1, tree_chunk = 1;  // walk schedule (nb_tree_schedule)
    float4 *tree_P = nullptr, *tree_Plo = nullptr;
    int *tree_perm = nullptr;
    double *tree_box = nullptr;

    // fast multipole scratch (on first use; node arrays follow the tree's capacity)
    nb::FmmView fmm{};
    int fmm_cap = 0;             // nodes the expansion arrays hold
    int fmm_np = 0;              // floats per expansion they hold

    // ORB and LET scratch (allocated on first use)
    unsigned long long *orb_buf = nullptr;  // boxes [ORB_MAX_P][6], then histograms [ORB_MAX_P/2][256]
    int *orb_perm = nullptr;                // [n_max] body order of a pack or an id sort
    nb::LetScratch let{};                   // per tree node (let_cap nodes)
    int let_cap = 0;
    float *let_box = nullptr;               // 6 floats out + 6 unsigned of work
    int *let_queue = nullptr;               // group queue of the LET walks
    nb::WalkSource *let_src = nullptr;      // [1 + WALK_MAX_MORE] the trees of one multi-tree walk
    double *let_tpart = nullptr;            // split LET walk: per-tree sums
    int *let_tcnt = nullptr;                //   per-tree counts
    unsigned *let_tctr = nullptr;           //   per-group arrivals (kept zero)
    int64_t let_tpart_cap = 0, let_tcnt_cap = 0, let_tctr_cap = 0;
    int64_t let_n = 0;                      // bodies of the local tree of nb_let_build

    std::map<const void *, int> occ;  // resident CTAs per SM, per kernel

    // event timing of pair-kernel launches (nb_profile)
    bool prof_on = false;
    struct ProfRec { int kind; cudaEvent_t a, b; };
    std::vector<ProfRec> prof;          // recorded launches
    std::vector<cudaEvent_t> ev_pool;   // free events
    int64_t launches = 0;
    std::string last_error;
};
