/*
 * nbody.h -- C ABI of libnbody.so, the GB300 (sm_103a) softened direct-sum
 * n-body force path.
 *
 * The operation (paper Sec. IV, "the n-body problem"; Sec. IV-B: the force
 * calculation takes upwards of 90% of the cycles):
 *
 *   a_i = G * sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^{3/2}
 *
 * summed exactly over all pairs (the paper's tree code, Sec. IV-A,
 * approximates this sum), plus the position/velocity update that consumes it
 * ("Move_bodies", Sec. IV-B pseudo-code) as a kick-drift-kick leapfrog.
 *
 * Conventions shared by every entry point:
 *   - Arrays are caller-owned DEVICE pointers on the context's device,
 *     contiguous, float64, 8-byte aligned: positions, velocities and
 *     accelerations are row-major (n,3) ("[n][3]"), masses (n).
 *   - Work is enqueued on the context's stream; no call synchronises unless
 *     its comment says so.  Inputs must stay valid until the stream reaches
 *     the work.
 *   - Arguments are checked on the host before anything is enqueued; a
 *     rejected call enqueues nothing and returns NB_EINVAL.
 *   - Errors are status codes; nb_last_error() gives the message.  No C++
 *     exception crosses this boundary.
 *   - Outputs are overwritten unless stated as accumulated.
 *   - G, eps and dt are float64 in every precision mode; eps >= 0.
 *     With eps == 0 the self pair is skipped explicitly; with eps > 0 it
 *     contributes exactly zero.
 *   - The library owns only scratch memory inside the context.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx; /* opaque, created and freed by the library */

typedef enum {
    NB_OK = 0,
    NB_EINVAL = 1,      /* bad argument (null/misaligned pointer, n out of range, NaN G ...) */
    NB_ECUDA = 2,       /* a CUDA runtime call failed (message holds its name and text) */
    NB_ENOMEM = 3,      /* device allocation failed or scratch too small */
    NB_ENONFINITE = 4,  /* a kernel produced a non-finite result (reported by nb_sync/nb_energy) */
    NB_ETIMEOUT = 5     /* reserved: no entry point waits on a device flag */
} nb_status;

typedef enum {
    NB_FP64 = 0,      /* every pair term and sum in float64; valid for any pair
                         whose r^2 + eps^2 is a positive normal float64 and whose
                         1/(r^2 + eps^2)^(3/2) does not overflow (e.g. eps = 0 and
                         separations from 1e-100 to 1e100) */
    NB_FP32 = 1,      /* float32 pair terms, one float32 running sum per body;
                         float32 modes need masses >= 0 (a negative mass can give
                         NB_ENONFINITE with the log-domain kernel variants) */
    NB_FP32_COMP = 2, /* float32 pair terms, float32 sums per j-tile added into
                         per-body Kahan-compensated (sum, carry) pairs */
    NB_DF64 = 3       /* float64 accuracy on the float32 pipe: every pair term in
                         double-float arithmetic (hi + lo float32 pairs formed with
                         error-free sums and products, ~48 significant bits), bodies
                         in Morton order with tile-local origins, float64 sums per
                         j-tile; forces, steps and rollouts (the adjoint and the
                         diagnostics run in float64, the batched kernel is
                         float32 only).  Pair terms carry float32's exponent
                         range: r^2 + eps^2 must lie within 1.2e-38 .. 3.4e38
                         (use NB_FP64 beyond it) */
} nb_precision;

/* Flags for nb_step / nb_rollout / nb_step_batched. */
#define NB_ACC_VALID 1u   /* acc already holds F(pos): skip the initial force evaluation */
#define NB_USE_GRAPH 2u   /* run the step loop as one captured CUDA graph */

/* Flags for nb_step_backward. */
#define NB_BWD_AT_END   1u  /* traj[nsteps] is the last state of the run */
#define NB_BWD_AT_START 2u  /* traj[0] is the first state of the run */

/*
 * Create a context on `device` for systems of up to n_max bodies in
 * precision `p`.  Work is enqueued on `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream).  Allocates the scratch (packed bodies, split
 * partials, reduction buffers) up front.  *out is NULL on failure.
 */
nb_status nb_create(nb_ctx **out, int64_t n_max, nb_precision p, int device,
                    void *cuda_stream);

/* Free the context and its scratch (synchronises its stream first).  NULL is a no-op. */
nb_status nb_destroy(nb_ctx *ctx);

/* Change the stream later work is enqueued on. */
nb_status nb_set_stream(nb_ctx *ctx, void *cuda_stream);

/* Message of the last failed call on this context (or of the last failed
 * nb_create when ctx is NULL).  Owned by the library; valid until the next call. */
const char *nb_last_error(const nb_ctx *ctx);

/* Wait for the context's stream; NB_ENONFINITE if any kernel flagged a
 * non-finite output since the last check (the flag is then cleared). */
nb_status nb_sync(nb_ctx *ctx);

/*
 * Accelerations a = F(pos, mass) (paper Sec. IV-A/IV-B force calculation,
 * as the exact all-pairs sum).  pos [n][3], mass [n], acc [n][3] (out).
 * 0 <= n <= n_max; n == 0 is a no-op.
 */
nb_status nb_forces(nb_ctx *ctx, int64_t n, const double *pos, const double *mass,
                    double G, double eps, double *acc);

/*
 * nsteps kick-drift-kick leapfrog steps of dt, in place on pos and vel (the
 * reading of "Move_bodies", paper Sec. IV-B):
 *   v += dt/2 a;  x += dt v;  a = F(x);  v += dt/2 a.
 * acc [n][3] is the force cache: on entry it must hold F(pos) if flags has
 * NB_ACC_VALID, otherwise it is computed first (nsteps + 1 force
 * evaluations); on return it holds F at the final positions.  The state
 * update is float64 in every precision mode.  nsteps >= 0.
 */
nb_status nb_step(nb_ctx *ctx, int64_t n, double *pos, double *vel, const double *mass,
                  double G, double eps, double dt, int64_t nsteps, double *acc,
                  unsigned flags);

/*
 * nb_step that also records the state every `record_every` steps (before
 * step 0, after step record_every, ...; the final state is recorded when
 * nsteps is a multiple of record_every): record r goes to rec_pos[r][n][3]
 * and, if rec_vel is not NULL, rec_vel[r][n][3].  The caller sizes them for
 * nsteps / record_every + 1 records.  record_every <= 0 records nothing.
 * Used for adjoint checkpoints and for recomputing a segment's trajectory.
 */
nb_status nb_rollout(nb_ctx *ctx, int64_t n, double *pos, double *vel, const double *mass,
                     double G, double eps, double dt, int64_t nsteps, double *acc,
                     unsigned flags, int64_t record_every, double *rec_pos,
                     double *rec_vel);

/*
 * Diagnostics in float64 (pair terms too, in every precision mode):
 * out_host[9] = {E_kin, E_pot, E_tot, P_x, P_y, P_z, F_x, F_y, F_z} with
 * E_kin = 1/2 sum m|v|^2, E_pot = -G sum_{i<j} m_i m_j / sqrt(r_ij^2+eps^2),
 * P = sum m v and F = sum m a (zero by Newton's third law).  out_host is
 * HOST memory; this call synchronises the stream and also reports
 * NB_ENONFINITE.  The paper reports no diagnostics; these are the standard
 * conserved quantities of the softened problem.
 */
nb_status nb_energy(nb_ctx *ctx, int64_t n, const double *pos, const double *vel,
                    const double *mass, double G, double eps, double *out_host);

/*
 * Vector-Jacobian product of the force map (no counterpart in the paper;
 * derived from the force formula).  With d_kj = x_j - x_k,
 * s = sqrt(|d|^2+eps^2) and K(d) = I/s^3 - 3 d d^T/s^5:
 *   grad_pos_k  = G sum_{j != k} K(d_kj) (m_k lam_j - m_j lam_k)
 *   grad_mass_k = G sum_{i != k} lam_i . (x_k - x_i) / s_ik^3
 * for lam = grad_acc [n][3] = dL/da.  grad_pos [n][3] and grad_mass [n] are
 * overwritten.  FP32 modes: float32 pair terms, float64 accumulation.
 */
nb_status nb_forces_backward(nb_ctx *ctx, int64_t n, const double *pos, const double *mass,
                             double G, double eps, const double *grad_acc,
                             double *grad_pos, double *grad_mass);

/*
 * Reverse sweep of nsteps leapfrog steps (no counterpart in the paper).
 * traj [nsteps+1][n][3] holds the positions x_0..x_nsteps of the segment
 * (from nb_rollout with record_every = 1).  lam_x, lam_v [n][3] hold on entry
 * the adjoints of the segment's final position and velocity, lam_m [n] the
 * mass adjoint so far; on return lam_x, lam_v hold the adjoints of the
 * segment's initial state and lam_m has the segment's contribution ADDED.
 * Per step, last to first: lam_v += dt lam_x (drift); the two half-kicks
 * that meet at a position x_s add VJP_F(x_s, dt lam_v) to (lam_x, lam_m).
 * Flags: NB_BWD_AT_END: traj[nsteps] is the end of the whole run, so its
 * closing half-kick VJP_F(x, dt/2 lam_v) is applied first; otherwise the
 * later segment already applied it.  NB_BWD_AT_START: traj[0] is the start
 * of the run, so the VJP there uses dt/2 instead of dt.  nsteps == 0 is a
 * no-op.
 */
nb_status nb_step_backward(nb_ctx *ctx, int64_t n, const double *traj, const double *mass,
                           double G, double eps, double dt, int64_t nsteps,
                           double *lam_x, double *lam_v, double *lam_m, unsigned flags);

/*
 * Batched independent systems (the paper's dynamic-chunk load balancing,
 * Sec. V-C / Table VI, applied to (system, i-tile) work items).
 * nb_batch_plan builds the work queue for nsys systems whose bodies are
 * concatenated, system k owning bodies [offsets[k], offsets[k+1]); offsets
 * is HOST memory with nsys + 1 entries, offsets[0] = 0, non-decreasing,
 * offsets[nsys] <= n_max.  Items are ordered largest cost first.  The plan
 * stays in the context until the next nb_batch_plan.
 */
nb_status nb_batch_plan(nb_ctx *ctx, int64_t nsys, const int64_t *offsets);

/* Forces of every planned system in one persistent launch.  Arrays cover all
 * offsets[nsys] bodies; bodies of different systems do not interact. */
nb_status nb_forces_batched(nb_ctx *ctx, const double *pos, const double *mass,
                            double G, double eps, double *acc);

/* nb_step over every planned system: one persistent force launch per step;
 * with NB_USE_GRAPH the whole loop is one CUDA graph launch (captured on
 * first use and cached per argument set). */
nb_status nb_step_batched(nb_ctx *ctx, double *pos, double *vel, const double *mass,
                          double G, double eps, double dt, int64_t nsteps, double *acc,
                          unsigned flags);

/*
 * Kernel variants and tuning (used by the autotuner).  kind: 0 = force,
 * 1 = batched force, 2 = force VJP; the variant tables depend on precision.
 * nb_variant_count -> number of compiled variants (0 if none);
 * nb_variant_info fills threads per CTA, bodies per thread and j-tile size.
 * nb_tune_set makes calls with lo <= n < hi use `variant`, with `split`
 * j-splits across CTAs (0 = chosen by the scheduler); later entries win.
 * For the batched kind, n is the planned bodies and `split` is the item-cap
 * divisor d (0 = 4): when a plan has more items than resident CTAs, a work
 * item holds at most 1/d of an even per-CTA share of the pairs; it takes
 * effect at the next nb_batch_plan.
 * variant < 0 clears the kind's table.  nb_tune_get reports the variant and
 * split a call with n bodies would use.
 */
int nb_variant_count(int kind, nb_precision p);
nb_status nb_variant_info(int kind, nb_precision p, int variant, int *threads,
                          int *bodies_per_thread, int *jtile);
nb_status nb_tune_set(nb_ctx *ctx, int kind, int64_t lo, int64_t hi, int variant, int split);
nb_status nb_tune_get(nb_ctx *ctx, int kind, int64_t n, int *variant, int *split);

/*
 * Body order of the float32 force kernels.  Each CTA forms pair differences
 * relative to the centre of its i-tile; with spatially compact i-tiles this
 * keeps close pairs accurate far from the origin.  mode 0: bodies in input
 * order; 1: always in Morton (Z-curve) order; 2 (default): Morton order when
 * n >= min_n (default 131072).  The order is recomputed (deterministically)
 * for every force evaluation; results are returned in input order.  No
 * effect on NB_FP64 contexts or on the batched kernel.
 */
nb_status nb_set_order(nb_ctx *ctx, int mode, int64_t min_n);

/* Number of kernels this context has launched so far (for launch accounting). */
int64_t nb_launch_count(const nb_ctx *ctx);

/*
 * Kernel timing with CUDA events recorded on the context's stream around
 * each pair-kernel launch (not inside captured graphs).  nb_profile(ctx, 1)
 * clears the record and starts recording, nb_profile(ctx, 0) stops.
 * nb_profile_read synchronises the stream and returns, for `kind`
 * (0 force, 1 batched force, 2 force VJP, 3 energy, 4 tree walk, 5 tree
 * build: sort, pack, levels, moments, 6 fast multipole upward and downward
 * passes, 7 fast multipole near field), the launches (sequences, for 5 to 7)
 * recorded and their summed duration in milliseconds.
 */
nb_status nb_profile(nb_ctx *ctx, int enable);
nb_status nb_profile_read(nb_ctx *ctx, int kind, int64_t *launches, double *total_ms);

/* Device properties the scheduler uses: SM count, and resident CTAs per SM
 * of the force kernel a call with n bodies would use. */
nb_status nb_device_info(nb_ctx *ctx, int64_t n, int *num_sms, int *ctas_per_sm);

/*
 * Barnes-Hut tree code (paper Sec. IV-A): the bodies are put in an octree by
 * dividing space 8 ways until a cell holds few enough bodies; a body meets a
 * cell that is distant enough as one particle of the cell's total mass at its
 * centre of mass, and otherwise the cell's children, down to the bodies of
 * nearby leaves.  The paper names neither an opening rule nor a threshold;
 * this library's reading:
 *   - space is the cube at the bodies' box minimum with edge `ext`, the
 *     longest box side; a body's cell at level L (edge ext / 2^L) is given by
 *     the top 3L bits of its 30-bit Morton key, q = floor((x - lo) 1024/ext)
 *     clamped to [0, 1023] per axis;
 *   - a cell is a leaf when it holds at most leaf_cap bodies or is at level 10;
 *   - bodies are taken `group` (32 or 64) at a time in key order, and the
 *     group walks the tree together: a cell acts as its monopole only when,
 *     for every body of the group, the float32 distance from the body to the
 *     cell's cube is at least edge / theta (theta = 0 opens every cell: the
 *     direct sum through the tree);
 *   - cell masses and centres of mass are float64; pair terms are float32 in
 *     coordinates relative to the group's centre, summed per 32 sources and
 *     folded into Kahan-compensated sums; acc is float64.
 * The tree is rebuilt on every call, fully on the device (no host
 * synchronisation, so nb_tree_step can run as one captured graph).
 *
 * nb_tree_forces: acc [n][3] (out).  theta >= 0 and finite; 1 <= leaf_cap <=
 * NB_TREE_MAX_LEAF; group 32 or 64 (64 shares each walk among more bodies:
 * faster, a little more conservative); counts (optional, int32 [n][2], 8-byte aligned) receives
 * per body the number of cells and of bodies (itself included) it met.
 * Any precision mode (the walk is float32 in each).  The first call (and a
 * call whose leaf_cap needs more nodes than any before) allocates the tree
 * scratch: 132 bytes per node for 1 + sum_{L=1..10} min(8^L, n_max,
 * 8 floor(n_max / (leaf_cap + 1))) nodes, a bound no tree exceeds (about
 * 2.3e6 nodes for n_max = 2^20, leaf_cap = 16), plus 40 bytes per body; this
 * synchronises the device and drops the context's captured graphs.  nb_sync
 * returns NB_ENOMEM if a tree ever outgrew its arrays (the build then stops a
 * level early; the bound rules it out).
 *
 * nb_tree_step: nb_step with tree forces (nsteps + 1 tree builds and walks,
 * the first skipped with NB_ACC_VALID); NB_USE_GRAPH runs the steps as one
 * captured graph.
 *
 * nb_tree_stats: {nodes, leaves, cell interactions, body interactions} of
 * the last tree force evaluation on the context (synchronises its stream).
 */
#define NB_TREE_MAX_LEAF 65536
nb_status nb_tree_forces(nb_ctx *ctx, int64_t n, const double *pos, const double *mass,
                         double G, double eps, double theta, int leaf_cap, int group,
                         double *acc, int32_t *counts);
nb_status nb_tree_step(nb_ctx *ctx, int64_t n, double *pos, double *vel, const double *mass,
                       double G, double eps, double theta, int leaf_cap, int group, double dt,
                       int64_t nsteps, double *acc, unsigned flags);
nb_status nb_tree_stats(nb_ctx *ctx, int64_t *out);

/*
 * How the tree walk deals its groups of bodies to warps, after the paper's
 * OpenMP loop schedules (Sec. II; Sec. V-C compares them on the tree code):
 * sched 0 static (one warp per group, a grid covering every group), 1
 * dynamic (the default: resident warps take `chunk` consecutive groups at a
 * time from an atomic counter), 2 guided (chunks of max(chunk, remaining /
 * (2 x warps))).  1 <= chunk <= 2^20 (default 1).  Results do not depend on
 * the schedule, only the time does.  Drops the context's captured graphs.
 */
nb_status nb_tree_schedule(nb_ctx *ctx, int sched, int chunk);

/*
 * Fast multipole method: the O(N) method the paper names as the successor of
 * its tree code (Sec. VI, after Greengard and Rokhlin).  The paper gives no
 * formulation; the one here (the same as the oracle's):
 *  - the Barnes-Hut tree above (same cube, keys, leaf rule, leaf_cap);
 *  - per cell a Cartesian Taylor expansion of order `order` (2..6) of the
 *    softened potential about the cube's centre: moments of the cell's
 *    bodies, local coefficients of the potential of its sources;
 *  - target cell A and source cell B are well separated when
 *    |z_A - z_B| >= (r_A + r_B) / theta, z the cube centre, r = sqrt(3)/2 of
 *    the edge (decided exactly on integer centres);
 *  - the pairs come from the dual-tree traversal from (root, root): a cell
 *    takes the candidates its parent handed down; separated -> B's expansion
 *    acts on A; both leaves -> the bodies interact directly; A a leaf -> B's
 *    children are candidates; B a leaf or smaller than A -> B is handed to
 *    A's children; else B's children are;
 *  - a body's acceleration is G times (the direct sum over the bodies of the
 *    leaves it meets directly, self pair excluded, plus the gradient of the
 *    local expansion of its leaf, which holds its ancestors' translated).
 * theta = 0 separates nothing: the direct sum.  The series converge for
 * theta < 1; the error falls with smaller theta and larger order.
 *
 * nb_fmm_forces: acc [n][3] (out).  theta >= 0 and finite; 2 <= order <= 6;
 * 1 <= leaf_cap <= 64.  counts (optional, int32 [n][3], 4-byte aligned)
 * receives per body the source cells acting on its leaf and the leaf's
 * ancestors, the bodies those cells hold, and the bodies it meets directly
 * (itself included); the last two sum to n.  Float32 arithmetic in every
 * precision mode, float64 output.  Allocates on first use (the tree scratch
 * of nb_tree_forces, plus 2 np + 18 4-byte words per tree node, np the
 * (order+1)(order+2)(order+3)/6 expansion coefficients rounded up to a
 * multiple of 4; a pool of candidate lists, 4 (2^20 + 32 n_max) bytes to start;
 * the cells' expansion lists, 132 (4096 + 2 n_max) bytes to start; and the
 * leaves' lists of directly summed cells, 260 (4096 + n_max / 4) bytes to
 * start).  Synchronises the context's stream at the end: if a list outgrew
 * its store, the store is doubled and the passes run again.
 * Non-finite results are reported by nb_sync.
 *
 * nb_fmm_stats: {nodes, leaves, cell-to-cell expansions, direct body pairs
 * (self pairs included)} of the last FMM evaluation on the context.
 */
#define NB_FMM_MIN_ORDER 2
#define NB_FMM_MAX_ORDER 6
#define NB_FMM_MAX_LEAF 64
nb_status nb_fmm_forces(nb_ctx *ctx, int64_t n, const double *pos, const double *mass, double G,
                        double eps, double theta, int order, int leaf_cap, double *acc,
                        int32_t *counts);
nb_status nb_fmm_stats(nb_ctx *ctx, int64_t *out);
/* nb_step with FMM forces: nsteps + 1 evaluations (the first skipped with
 * NB_ACC_VALID), the closing half-kick fused into the kernel that writes the
 * accelerations.  Synchronises like nb_fmm_forces, so NB_USE_GRAPH is
 * refused (NB_EINVAL). */
nb_status nb_fmm_step(nb_ctx *ctx, int64_t n, double *pos, double *vel, const double *mass,
                      double G, double eps, double theta, int order, int leaf_cap, double dt,
                      int64_t nsteps, double *acc, unsigned flags);
/* Replace the candidate pool by one of `entries` ints (1 <= entries < 2^31),
 * and the stores of the cells' expansion lists and of the leaves' lists of
 * directly summed cells by entries / 32 + 1 chunks of 32 each, e.g. to size
 * them for a known workload; synchronises the stream.  A store too small
 * still gives the same results: the passes grow it and run again. */
nb_status nb_fmm_reserve(nb_ctx *ctx, int64_t entries);

/*
 * Parallel tree code over P processors (paper Sec. IV-B): orthogonal
 * recursive bisection (ORB) of space into P equal-count domains, a tree per
 * processor over its own bodies, and locally essential trees (LET): each
 * processor sends every other the part of its tree that the other's bodies
 * need, then computes its bodies' forces as in the sequential code.  These
 * calls are one processor's share; the collectives between them (sums,
 * min/max, all-to-all exchanges) belong to the caller's communicator.
 *
 * ORB.  A part shared by p processors is cut across the longest side of its
 * bounding box; the lower part takes floor(p/2) processors and the
 * k = floor(count floor(p/2) / p) bodies first in (coordinate, body id)
 * order.  A part is named by its first processor (a "group"); group arrays
 * are device int32 [n], initially all 0, and after the last cut hold each
 * body's processor.  ids are device int64 [n], unique over all processors,
 * in [0, 2^31).  The cut is found without moving bodies by a radix select
 * on the 96-bit key (order-preserving image of the float64 coordinate, the
 * 32-bit id), eight bits per round, rounds 0..11 most significant first.
 *  nb_orb_box: per group g < ngroups (<= NB_ORB_MAX_P), box_out[g] =
 *    {min xyz, max xyz} of this processor's bodies of g (HOST, float64;
 *    +inf/-inf when it has none).  Synchronises.
 *  nb_orb_hist: for the nactive (<= NB_ORB_MAX_P / 2) parts being cut,
 *    active[r] = the part's group, axis[r] in {0,1,2} its cut axis and
 *    prefix[2r], prefix[2r+1] the key bits (high 64, low 32) fixed so far:
 *    hist_out[r][d] (HOST int64) = this processor's bodies of the part whose
 *    key starts with the first 8 round bits of the prefix and has digit d
 *    next.  Synchronises.
 *  nb_orb_cut: bodies of active part r whose key is not below the split
 *    key (split[2r], split[2r+1]) move to group upper[r] (> active[r]).
 *  nb_orb_pack: the bodies ordered by rank (stable), into the *_out device
 *    arrays, and counts_out[r] (HOST) bodies per rank r < P; the send
 *    buffers of an all-to-all exchange.  Synchronises.
 *  nb_orb_order: the bodies ordered by id (after an exchange, so that each
 *    processor's tree and groups do not depend on the exchange's order).
 * LET.
 *  nb_let_build: the tree of nb_tree_forces (readings of that call) over
 *    this processor's n bodies, kept in the context until the next tree-code
 *    or FMM call on it (after which nb_let_export and nb_let_forces refuse
 *    until nb_let_build runs again); box_out (HOST, 6
 *    floats) = the float32 box {min xyz, max xyz} of the bodies, which the
 *    other processors need for their LETs.  Synchronises.
 *  nb_let_export: the LET of the local tree for a destination whose bodies
 *    lie in the float32 box (HOST, 6 floats, from its nb_let_build): the
 *    root is sent; a sent node distant enough from the box (the walk's
 *    opening test, so every body inside accepts it) goes alone; otherwise a
 *    sent leaf goes with its bodies and a sent cell with all its children.
 *    *size_out receives the LET's size in bytes; with out == NULL only the
 *    size is computed, otherwise out (device, 16-byte aligned, capacity
 *    bytes; NB_ENOMEM if too small) receives the LET, a self-contained
 *    buffer to send as bytes.  Synchronises once.
 *  nb_let_forces: acc [n][3] (device, the bodies of nb_let_build in their
 *    order) = G times the walk of the local tree plus the walks of the nlet
 *    received LETs (lets: HOST array of device pointers, 16-byte aligned, in
 *    the order to add them), with groups of `group` (32 or 64) bodies and
 *    the opening angle theta of the exports; counts (optional, device int32
 *    [n][2]) = cells and bodies met over all trees.  With no LET it is the
 *    tree code's nb_tree_forces.  nb_tree_stats then reports the summed
 *    interactions.  Up to 64 trees are walked in one launch, one task per
 *    (group of bodies, tree), the group's float64 sums added in tree order;
 *    the context keeps per-tree sums for that (24 bytes per body and tree,
 *    grown on demand).
 */
#define NB_ORB_MAX_P 64
nb_status nb_orb_box(nb_ctx *ctx, int64_t n, const double *pos, const int32_t *group, int ngroups,
                     double *box_out);
nb_status nb_orb_hist(nb_ctx *ctx, int64_t n, const double *pos, const int64_t *id,
                      const int32_t *group, int nactive, const int32_t *active,
                      const int32_t *axis, const uint64_t *prefix, int round, int64_t *hist_out);
nb_status nb_orb_cut(nb_ctx *ctx, int64_t n, const double *pos, const int64_t *id,
                     int32_t *group, int nactive, const int32_t *active, const int32_t *axis,
                     const uint64_t *split, const int32_t *upper);
nb_status nb_orb_pack(nb_ctx *ctx, int64_t n, const int32_t *rank, int P, const double *pos,
                      const double *vel, const double *mass, const int64_t *id, double *pos_out,
                      double *vel_out, double *mass_out, int64_t *id_out, int64_t *counts_out);
nb_status nb_orb_order(nb_ctx *ctx, int64_t n, const double *pos, const double *vel,
                       const double *mass, const int64_t *id, double *pos_out, double *vel_out,
                       double *mass_out, int64_t *id_out);
nb_status nb_let_build(nb_ctx *ctx, int64_t n, const double *pos, const double *mass, int leaf_cap,
                       float *box_out);
nb_status nb_let_export(nb_ctx *ctx, double theta, const float *box, void *out, int64_t capacity,
                        int64_t *size_out);
nb_status nb_let_forces(nb_ctx *ctx, double G, double eps, double theta, int group, int64_t nlet,
                        const void *const *lets, double *acc, int32_t *counts);

/*
 * nb_forces_noalloc -- accelerations as nb_forces in the NB_FP32_COMP form
 * (float32 pair terms, Kahan-compensated per-tile sums, float64 output), for
 * callers that cannot allocate device memory: code whose device memory is
 * owned by another allocator (a framework's pool that must account for every
 * byte) or capped by a fixed budget, and latency-critical loops in which a
 * cudaMalloc could block or synchronise the device.  The paper has no
 * counterpart; this is a service of the library.
 *
 * It allocates nothing: no context, no cudaMalloc/cudaFree.  Its scratch
 * (packed bodies, split partials, counters; about 8 MiB) is one fixed
 * __device__ array that every GPU loading the library holds until the
 * process exits, which bounds n to NB_NOALLOC_MAX_BODIES.  Work runs in the
 * calling thread's current CUDA context and device, enqueued on
 * `cuda_stream` (NULL = legacy default stream); pos [n][3], mass [n] and
 * acc [n][3] are device arrays of that device, acc is overwritten.  Bodies
 * are processed in input order (no spatial sort).
 *
 * The first call in each CUDA context does a one-time set-up: it looks up
 * the scratch array's device address in that context (cudaGetSymbolAddress)
 * and keeps it, keyed by the context; make that first call before any stream
 * capture.  Every call in a context shares the one scratch array and it keeps
 * the last call's contents: each call clears the counters and the error word
 * it uses before its kernels run, and calls whose work overlaps on the GPU
 * (different streams without ordering, several threads) race and give wrong
 * results; order them on one stream.
 *
 * Returns NB_EINVAL (n < 0, n > NB_NOALLOC_MAX_BODIES, NULL/misaligned/
 * non-device arrays, non-finite G, eps < 0) before enqueuing anything,
 * NB_ECUDA if the runtime fails or no CUDA context is current; there is no
 * message text.  It never returns NB_ENONFINITE: with no context to hold an
 * error word that a later call could read, non-finite accelerations are not
 * reported, so check acc when the inputs may hold infinities or NaNs.  n == 0
 * is a no-op.
 */
#define NB_NOALLOC_MAX_BODIES 65536
nb_status nb_forces_noalloc(int64_t n, const double *pos, const double *mass, double G,
                            double eps, double *acc, void *cuda_stream);

/*
 * Host-only scheduling helpers (no GPU needed; exported for tests).
 *
 * nb_choose_split: number of j-splits for n_itiles i-tiles of tile_bodies
 * bodies over n_jtiles j-tiles on `slots` resident CTAs, maximising
 * (items / slots) / ceil(items / slots) times a per-item overhead factor,
 * with nsplit * n_itiles * tile_bodies <= max_split_bodies.
 *
 * nb_plan_batch_host: the work items of the batched kernel for CTAs of
 * `threads` x `bodies_per_thread` bodies and j-tiles of `jtile`, largest
 * cost first.  Each system gets the most lanes per body that still cover it
 * with one item, and more while an item would exceed max_item_pairs
 * (0 = no cap).  items_out holds 8 int32 per item {i0, i_end, j0, j1,
 * lanes, sys, 0, 0}; returns the item count (items_out may be NULL to
 * count), or -1 for invalid offsets or when more than max_items are needed.
 */
int nb_choose_split(int64_t n_itiles, int64_t n_jtiles, int64_t slots,
                    int64_t max_split_bodies, int64_t tile_bodies);
int64_t nb_plan_batch_host(int64_t nsys, const int64_t *offsets, int threads,
                           int bodies_per_thread, int jtile, int64_t max_item_pairs,
                           int32_t *items_out, int64_t max_items);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
