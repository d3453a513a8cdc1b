/*
 * fmm.h -- C ABI of libfmm_gb300.so, a GB300-native (sm_103a) implementation of the
 * asymmetric adaptive 2D fast multipole method of S. Engblom, "On well-separated sets and fast
 * multipole methods".
 *
 * The library evaluates, for N points z_i = (x_i, y_i) with strengths q_i,
 *
 *     phi_i = sum_{j != i} q_j log|z_i - z_j|            (Eq. (1.1), 2D harmonic kernel)
 *
 * with the paper's method (Section 4): a balanced tree obtained by splitting every box at the
 * median along x and then along y (Fig. 1.1, Fig. 4.1), strong/weak interaction lists from the
 * one-parameter theta-criterion (Criterion 2.1), order-p complex expansions pushed through
 * P2M -> M2M -> M2L -> L2L -> L2P, and a direct near-field sum along the finest strong lists.
 *
 * Conventions shared by every entry point
 *   - Array arguments are DEVICE pointers (cudaMalloc'd or equivalent, on the device that is
 *     current when the call is made) unless the argument name ends in _host.  They are owned by
 *     the caller and are not retained after the call returns.
 *   - Handles (fmm_tree, fmm_lists) are owned by the library; release them with the matching
 *     *_destroy function.  A handle is bound to the device that was current at creation.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Compute calls only enqueue
 *     work on it and return; they never synchronise with the host.  Conditions that can only
 *     be seen on the device (non-finite input, list capacity overflow) set a device-side status
 *     word that fmm_sync_status() reads.
 *   - Every int-returning function returns FMM_OK (0) or a negative fmm_status; the message of
 *     the last error on the calling thread is available from fmm_last_error().
 *   - There is no CPU fallback: every step runs in the library's CUDA kernels.
 *   - Point indices are 32-bit (N < 2^31).
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM_OK = 0,
    FMM_ERR_ARG = -1,        /* bad argument (null pointer, size, p, theta, ...)            */
    FMM_ERR_NONFINITE = -2,  /* a coordinate or strength is NaN or infinite                 */
    FMM_ERR_LEVELS = -3,     /* N < 4^levels: some leaf would be empty                      */
    FMM_ERR_OOM = -4,        /* device allocation failed                                    */
    FMM_ERR_CUDA = -5,       /* a CUDA runtime call failed                                  */
    FMM_ERR_CAPACITY = -6,   /* interaction lists exceeded the capacity of the fmm_lists   */
    FMM_ERR_TIMEOUT = -7,    /* a bounded device-side wait gave up                          */
    FMM_ERR_STATE = -8,      /* handle used out of order (e.g. lists of another tree)       */
    FMM_ERR_DEGENERATE = -9  /* field only: a leaf box of zero size (its points all coincide) */
} fmm_status;

typedef enum {
    FMM_MODE_FP64 = 0,   /* every stage in binary64                                         */
    FMM_MODE_MIXED = 1,  /* binary32 expansions, near field and accumulation (see below)    */
    FMM_MODE_SPLIT = 2   /* binary64 expansions (P2M .. L2P); the near field in float-float
                            (pairs of binary32: terms and sums, about 2^-46 relative); far and
                            near joined in binary64 */
} fmm_mode;

typedef struct fmm_tree_s* fmm_tree;
typedef struct fmm_lists_s* fmm_lists;

/*
 * Parameters of one evaluation.
 *   p      expansion order: coefficients k = 0..p (a_0 is the logarithmic term), 0 <= p <= 40.
 *          The relative error behaves like theta^(p+1)/(1-theta)^2 (Section 3).
 *   mode   FMM_MODE_FP64, FMM_MODE_MIXED or FMM_MODE_SPLIT.
 *   tol    requested relative tolerance (0 = none).  In FMM_MODE_MIXED a tol below 1e-7 is
 *          beyond what binary32 expansions can deliver (their rounding alone is about 1e-7 of
 *          the potential), so such a call runs as FMM_MODE_SPLIT: binary64 expansions and a
 *          float-float near field, the accuracy of FMM_MODE_FP64 (the binary64 field, which
 *          has no split form, runs every stage in binary64).  Ignored in the other modes.
 */
typedef struct {
    int p;
    int mode;
    double tol;
} fmm_params;

/* ---------------------------------------------------------------------------------------------
 * Tree: Section 4 (median splits), Fig. 1.1, Fig. 4.1.
 * Box i of level l (0 <= l <= levels) has global id (4^l - 1)/3 + i; its children are boxes
 * 4i+k of level l+1 with k = 0:(x-low,y-low) 1:(x-low,y-high) 2:(x-high,y-low) 3:(x-high,y-high).
 * A set of n points is split along x into the floor(n/2) smallest in (x, input index) order and
 * the rest; each half is then split the same way along y.  The split coordinate is 0.5*(a+b)
 * of the two straddling coordinates.  The root is the tight bounding box of the points.
 * ------------------------------------------------------------------------------------------- */

/* Allocate a tree for n points and `levels` levels below the root (n >= 4^levels, levels <= 13,
 * n < 2^31).  Allocates device memory (synchronous); no kernel runs. */
int fmm_tree_create(int64_t n, int levels, fmm_tree* out);

/* Batched problems (no paper counterpart: the paper treats one point set at a time).
 * A tree may hold a forest of n_inst independent instances, instance i with n[i] points and
 * levels[i] levels (host arrays; each instance obeys the limits of fmm_tree_create, and the
 * total number of points is below 2^31).  Every call on such a tree processes all instances in
 * the same launches, each exactly as if it were alone: the points of instance i never interact
 * with those of another.  Point arrays (x, y, q, phi, perm) are the instances' arrays
 * concatenated in instance order; box arrays (rects) the instances' boxes concatenated (each in
 * its own global id order); leaf_begin the instances' 4^levels[i] + 1 offsets concatenated.
 * Indices stored in these arrays are local to their instance.  fmm_tree_instance reports where
 * instance i starts.  fmm_tree_create(n, L, out) is the forest of one instance. */
#define FMM_MAX_INSTANCES 65535
int fmm_tree_create_batched(int n_inst, const int64_t* n_host, const int* levels_host, fmm_tree* out);

/* Number of instances of a tree (or a negative fmm_status). */
int fmm_tree_num_instances(fmm_tree t);

/* Instance i of a tree (host values, any pointer may be NULL): its first point p0 and point
 * count n, levels, first box b0 and box count nbox, first leaf_begin entry lb0. */
int fmm_tree_instance(fmm_tree t, int i, int64_t* p0, int64_t* n, int* levels, int64_t* b0,
                      int64_t* nbox, int64_t* lb0);

/* Build the tree of points (x[n], y[n]) (binary64, device).  The tree keeps its own copy of
 * everything it needs; x and y may be reused after the work on `stream` completes.  Non-finite
 * coordinates set FMM_ERR_NONFINITE in the device status. */
int fmm_build_tree(fmm_tree t, const double* x, const double* y, void* stream);

/* The uniform-grid mesh in place of the median tree (no paper formula: the non-adaptive mesh
 * that Section 5 compares the adaptive code with).  The root is the square on the points'
 * bounding-box lower-left corner whose side is the box's longer side; every box splits into four
 * equal quadrants, children numbered as by fmm_build_tree; a point's leaf cell is
 * floor(((x - x0) / side) * 2^L), clamped, likewise in y; points are ordered by leaf, then by
 * input index.  Leaves may be empty or hold any number of points.  Lists, evaluation and export
 * then work on this mesh unchanged.  root_host (may be NULL): a given root square
 * {x0, y0, side} (host array of 3, side >= 0) used for every instance instead of the bounding
 * square, e.g. the unit square of Section 5's experiment; points outside it are clamped into its
 * edge cells.  Reads the largest leaf of every instance back to the host, so the call
 * synchronises `stream`; a later fmm_build_tree restores the median tree. */
int fmm_build_tree_uniform(fmm_tree t, const double* x, const double* y, const double* root_host, void* stream);

/* Copy the tree out (device pointers, any may be NULL):
 *   perm[n]            canonical point order: leaves in id order, inside a leaf ascending input
 *                      index; perm[k] is the input index of the k-th point.
 *   rects[4*nbox]      (x0, x1, y0, y1) per box in global id order, nbox = (4^(levels+1)-1)/3.
 *   leaf_begin[4^levels + 1]  leaf i holds perm[leaf_begin[i] .. leaf_begin[i+1]).        */
int fmm_tree_export(fmm_tree t, int32_t* perm, double* rects, int32_t* leaf_begin, void* stream);

/* Number of points, levels and boxes of a tree (host values; for a forest the totals over its
 * instances and the largest levels). */
int fmm_tree_info(fmm_tree t, int64_t* n, int* levels, int64_t* nbox);

void fmm_tree_destroy(fmm_tree t);

/* ---------------------------------------------------------------------------------------------
 * Tree construction that allocates nothing.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code inside an application whose own
 * memory manager owns the device (an allocation behind its back can fail or fragment what it
 * manages), or latency-critical loops that cannot take the device-wide synchronisation a
 * cudaMalloc/cudaFree may cause.  It computes exactly what fmm_build_tree
 * followed by fmm_tree_export computes, but every intermediate buffer lives in one fixed device
 * array compiled into the library (about 7.7 MB, held on every GPU that loads the library until
 * the process exits), so inputs are limited to n <= FMM_NOALLOC_MAX_POINTS points and
 * levels <= FMM_NOALLOC_MAX_LEVELS.
 *
 *   x[n], y[n]         point coordinates (binary64, device)
 *   perm[n]            output, as fmm_tree_export
 *   rects[4*nbox]      output, nbox = (4^(levels+1)-1)/3, as fmm_tree_export
 *   leaf_begin[4^levels + 1]  output, as fmm_tree_export
 *   status             optional (NULL or one device int32): receives the device status word of
 *                      the build (0, or FMM_ERR_NONFINITE's bit 1 for non-finite coordinates)
 *
 * Returns FMM_ERR_ARG for sizes beyond the limits (nothing is launched) and FMM_ERR_LEVELS when
 * n < 4^levels.  It calls no cudaMalloc, cudaFree or other allocating routine.  All calls share
 * the one array, so calls on the same device must not overlap in time (two streams or two host
 * threads running it at once corrupt each other's results).  The first call on a device looks
 * up the array's address (cudaGetSymbolAddress) and sets the tree kernels' shared-memory limit
 * (cudaFuncSetAttribute); make that first call before any stream capture.  Both are kept for the
 * life of the process, so after cudaDeviceReset (a new context) do not call it on that device
 * again.  Each of rects and leaf_begin must hold the element count above: the library cannot
 * check the length of a raw pointer.
 * ------------------------------------------------------------------------------------------- */
#define FMM_NOALLOC_MAX_POINTS 65536
#define FMM_NOALLOC_MAX_LEVELS 7

int fmm_build_tree_noalloc(const double* x, const double* y, int64_t n, int levels,
                           int32_t* perm, double* rects, int32_t* leaf_begin, int32_t* status,
                           void* stream);

/* ---------------------------------------------------------------------------------------------
 * Interaction lists: Section 4 with Criterion 2.1.
 * S(root) = {root}, W(root) = {}.  For a box b of level l >= 1 the candidates are the children
 * of every box of S(parent(b)) in ascending id; a candidate c joins W(b) when
 *     R + theta*r <= theta*d   and   R + r < d
 * (d = distance of the centres, R/r = larger/smaller radius; centre = rectangle midpoint,
 * radius = half diagonal), otherwise S(b).  Lists are CSR over global box ids whose entries are
 * within-level box indices in ascending order.  M2L runs along W on every level, the direct
 * near-field sum along S of the finest level.
 * ------------------------------------------------------------------------------------------- */

/* Allocate list storage for tree t with room for weak_capacity weak and strong_capacity strong
 * entries in total (0 = a default of 64 and 32 per box).  For a forest the totals are shared out
 * over the instances in proportion to their box counts (at least 16 weak and 8 strong per box). */
int fmm_lists_create(fmm_tree t, int64_t weak_capacity, int64_t strong_capacity, fmm_lists* out);

/* List storage of a forest with the capacity of every instance given (host arrays of n_inst
 * positive entries). */
int fmm_lists_create_batched(fmm_tree t, const int64_t* weak_capacity_host,
                             const int64_t* strong_capacity_host, fmm_lists* out);

/* Optional structural optimisations of Section 4; mode is a combination of the bits below
 * (FMM_LISTS_PLAIN = 0 is the default).
 *  FMM_LISTS_PARENTS: a box whose weak list holds all four children of a box P of the level
 *    above, as four consecutive entries 4k .. 4k+3, interacts with P instead whenever the
 *    theta-criterion between P and the box holds.  Such an entry is k | FMM_PARENT_FLAG (a
 *    within-level index of the level above).
 *  FMM_LISTS_EXCHANGE: at the finest level, a strongly coupled pair of leaves of different radii
 *    for which the criterion holds with the roles of r and R exchanged (r + theta*R <= theta*d,
 *    disjoint circles) leaves the strong list of the target for its exchange list: if the target
 *    is the smaller leaf the source's points are added to its local expansion (P2L), else the
 *    source's multipole expansion is evaluated at its points (M2P; entry s | FMM_SWAP_M2P).
 * Setting the mode allocates (synchronous) and requires a rebuild of the lists.  The exchange
 * lists share the strong capacity (their count is checked against it). */
#define FMM_LISTS_PLAIN 0
#define FMM_LISTS_PARENTS 1
#define FMM_LISTS_EXCHANGE 2
#define FMM_PARENT_FLAG 0x40000000
#define FMM_SWAP_M2P 0x20000000
int fmm_lists_set_mode(fmm_lists l, int mode);

/* Instance i's exchange lists (FMM_LISTS_EXCHANGE): xoff[nbox_i + 1] offsets over all its boxes
 * in level order (empty below the finest level), xidx[xoff[nbox_i]] within-level leaf indices
 * (| FMM_SWAP_M2P where the target is the larger leaf).  Device buffers; either may be NULL.
 * Synchronises the stream; *count_host (may be NULL) receives the number of entries. */
int fmm_lists_export_exchange(fmm_lists l, int i, int32_t* xoff, int32_t* xidx, int64_t* count_host,
                              void* stream);

/* Build the lists of tree t (which must have been built on the same stream or be complete)
 * for 0 < theta < 1.  Overflow of the capacity sets FMM_ERR_CAPACITY in the device status;
 * later kernels then read only within the capacity. */
int fmm_interaction_lists(fmm_tree t, fmm_lists l, double theta, void* stream);

/* Wait for `stream`, then report the list totals over all instances (host values, may be NULL)
 * and the status: FMM_ERR_CAPACITY when an instance's lists did not fit. */
int fmm_lists_sync(fmm_lists l, void* stream, int64_t* n_weak, int64_t* n_strong);

/* As fmm_lists_sync, with the entry counts of every instance (host arrays of n_inst entries,
 * may be NULL).  For an instance whose lists fit they are exact; for one that overflowed they
 * are a lower bound of what it needs (levels below the overflow see truncated lists). */
int fmm_lists_counts(fmm_lists l, void* stream, int64_t* n_weak_host, int64_t* n_strong_host);

/* Copy the lists out (device pointers): woff/soff[nbox+1], widx[n_weak], sidx[n_strong].
 * Trees of one instance only. */
int fmm_lists_export(fmm_lists l, int32_t* woff, int32_t* widx, int32_t* soff, int32_t* sidx,
                     void* stream);

/* The lists of instance i, as fmm_lists_export for that instance alone (nbox = its box count,
 * offsets start at 0). */
int fmm_lists_export_instance(fmm_lists l, int i, int32_t* woff, int32_t* widx, int32_t* soff,
                              int32_t* sidx, void* stream);

/* Lists of instance i from device arrays in the layout fmm_lists_export_instance writes (offsets
 * over the instance's boxes, within-level entries; weak entries may carry FMM_PARENT_FLAG): for
 * resuming from saved lists without rebuilding them.  Synchronises `stream` (reads the counts);
 * FMM_ERR_CAPACITY if they exceed the instance's capacities, FMM_ERR_STATE for lists with
 * exchange lists (FMM_LISTS_EXCHANGE).  Imported lists are not checked: call fmm_validate
 * before evaluating them. */
int fmm_lists_import(fmm_lists l, int i, const int32_t* woff, const int32_t* widx, const int32_t* soff,
                     const int32_t* sidx, void* stream);

/* Structural checks of a built tree and (if l is not NULL) its lists: leaf offsets from 0 to n,
 * the canonical order a permutation, every point inside its leaf's offsets, finite rectangles
 * and radii, list offsets non-decreasing within the capacities, every entry listed under its
 * target and within its level (parent entries within the level above, exchange entries within
 * the leaves).  Every read is in range, so corrupted structures are reported, not read out of
 * bounds.  Synchronises `stream`; FMM_OK, or FMM_ERR_STATE naming the first failing check. */
int fmm_validate(fmm_tree t, fmm_lists l, void* stream);

/* Failure-path self-test of the device's bounded waits (no paper counterpart): one warp runs
 * the wait the tensor-core M2L uses on an mbarrier that nothing completes; after `tries` tries
 * (1 .. 2^20) it gives up, records FMM_ERR_TIMEOUT in its status word and returns, leaving the
 * context usable.  Synchronises `stream`; returns FMM_ERR_TIMEOUT (the expected outcome). */
int fmm_selftest_bounded_wait(int64_t tries, void* stream);

/* Failure-path self-test of the work queues (no paper counterpart).  The upward pass (M2M of
 * every level of every instance) runs as one persistent launch over a queue of items in
 * dependency order; an item waits, bounded, until the items of the level below are counted done.
 * This runs that launch with instance 0's item count of its deepest M2M level raised by one, so
 * the level above waits for an item that is not in the queue: each such wait gives up after
 * `tries` tries (1 .. 2^20) and records FMM_ERR_TIMEOUT, and the launch completes.  Scratch
 * coefficients and status; the tree is unchanged and evaluates normally afterwards.  Needs an
 * instance 0 of at least 3 levels; synchronises `stream`; returns FMM_ERR_TIMEOUT (the expected
 * outcome). */
int fmm_selftest_queue_timeout(fmm_tree t, int64_t tries, void* stream);

void fmm_lists_destroy(fmm_lists l);

/* ---------------------------------------------------------------------------------------------
 * Evaluation: the upward pass (P2M on the leaves, M2M towards the root), M2L along the weak
 * lists of every level, the downward pass (L2L), L2P and the direct sum along the strong lists
 * of the finest level (Section 4).  Expansions are the classical complex ones of Section 5:
 * multipole a_0 log(z - c) + sum_k a_k (z - c)^-k, local sum_l b_l (z - c)^l, stored scaled by
 * the box radius.  phi[n] (binary64, device) receives the potentials in INPUT order.
 * q[n]: strengths (binary64, device).  The first call with a given p allocates the expansion
 * workspace of the tree (synchronous); later calls with the same or a smaller p allocate
 * nothing.
 * ------------------------------------------------------------------------------------------- */
int fmm_evaluate(fmm_tree t, fmm_lists l, const double* q, const fmm_params* prm, double* phi,
                 void* stream);

/* One whole step on new coordinates and strengths: fmm_build_tree, fmm_interaction_lists and
 * fmm_evaluate in one call, with the independent parts overlapped on a second stream owned by the
 * tree.  The lists of each level are built there as soon as the tree build has that level's box
 * geometry (beside the remaining partitions of the tree, then beside the packing and upward pass
 * on `stream`), and in the mixed mode the near field runs there while `stream` finishes the far
 * field.  Every
 * dependency goes through events, so the call may be captured into a CUDA graph on `stream`
 * (the first call creates the stream and its events: make it before capturing).  Same arguments
 * and errors as the three calls. */
int fmm_step(fmm_tree t, fmm_lists l, const double* x, const double* y, double theta, const double* q,
             const fmm_params* prm, double* phi, void* stream);

/* Launch-shape tuning (no paper counterpart).  The M2L and near-field launches of a tree use a
 * total number of blocks that is shared out over its instances in proportion to their work.
 * fmm_autotune runs complete evaluations of (t, l, q, prm) on `stream` for a ladder of such
 * totals, timing each with CUDA events, and keeps the fastest for later evaluations of this tree;
 * phi receives the potentials of the last run.  It synchronises with the host (not for use under
 * stream capture).  The chosen totals are reported in m2l_blocks / p2p_blocks (host, may be
 * NULL).  For the mixed path it also times the two binary32 M2L kernels (fmm_set_m2l_kernel)
 * with their tile shapes and the near field's targets per lane (fmm_set_near_shape), and keeps
 * the fastest.  fmm_set_launch sets the totals directly (0 = the built-in default); it
 * uploads small launch tables and so also synchronises.  Both replace the tree's launch tables
 * and grid sizes: a CUDA graph captured before either call still names the old ones and must
 * not be launched again; capture it anew. */
int fmm_autotune(fmm_tree t, fmm_lists l, const double* q, const fmm_params* prm, double* phi,
                 void* stream, int* m2l_blocks_host, int* p2p_blocks_host);
int fmm_set_launch(fmm_tree t, int m2l_blocks, int p2p_blocks);

/* Which kernel performs the binary32 M2L of tree t: 2 the tensor cores (tcgen05, split-tf32
 * products: each operand as a tf32 high and low part, three products accumulated in binary32;
 * p <= 31 only), 1 the SIMT units in plain binary32, 0 (default) by the order: tensor cores for
 * 23 <= p <= 31, SIMT units otherwise (on GB300 the tensor cores measured twice as fast at
 * p = 30 and 20% slower at p = 20).  Changing
 * the kind does not touch the launch tables, but a captured graph keeps the kernel it saw.
 * fmm_autotune sets 1 or 2 by timing both.  The binary64 path always uses the SIMT units. */
int fmm_set_m2l_kernel(fmm_tree t, int kind);
/* The current choice (0, 1 or 2), or a negative fmm_status. */
int fmm_get_m2l_kernel(fmm_tree t);

/* Tile shape of the tensor-core M2L (no paper counterpart).  chunk: every row of its 128-row
 * tiles takes `chunk` consecutive weak entries, one per tile, and keeps the sums of their common
 * targets in registers, so a larger chunk means fewer atomic flushes and a coarser split of the
 * entries over the blocks; 1 .. 256, or 0 for the built-in default (16).  stages: 2 = two TMEM
 * accumulator buffers, the epilogue of one tile overlapping the MMAs of the next (two blocks per
 * SM); 1 = one buffer, the epilogue after its own tile's MMAs (three blocks per SM up to p = 20);
 * 0 = by order (2 from p = 21 on).  fmm_autotune chooses both with the block count.
 * fmm_get_m2l_shape reports them (host pointers, may be NULL). */
int fmm_set_m2l_shape(fmm_tree t, int chunk, int stages);
int fmm_get_m2l_shape(fmm_tree t, int* chunk, int* stages);

/* Work shape of the binary32 near field for leaves of at most 64 points (no paper counterpart):
 * every lane takes `targets` points of a target leaf (2 or 4) against each source leaf, so each
 * source point it loads serves that many pair evaluations and the per-leaf-pair set-up is shared
 * by as many; 0 = the built-in default (2).  fmm_autotune chooses it with the block count.
 * fmm_get_near_shape reports it (host pointer, may be NULL). */
int fmm_set_near_shape(fmm_tree t, int targets);
int fmm_get_near_shape(fmm_tree t, int* targets);

/* ---------------------------------------------------------------------------------------------
 * Throughput probes (no paper counterpart): the peaks of the units the ALU-bound kernels use,
 * measured instead of derived.  fmm_probe_throughput launches one probe on `stream`: kind 0
 * binary32 FFMA, 1 the approximate base-2 logarithm (lg2.approx, the special-function unit), 2
 * binary64 DFMA; `iters` (1 .. 2^20) x 128 dependent operations per thread in 8 independent
 * chains, fmm_probe_blocks() blocks of 256 threads (8 per SM).  *ops (host) receives the
 * operations it performs (flop for the FMA probes, logarithms for kind 1); the caller times the
 * launch with events on the same stream.  out: device float buffer of fmm_probe_blocks() * 256
 * entries, written so that the work is not optimised away.  Asynchronous; FMM_ERR_ARG for a
 * bad kind or count.
 * ------------------------------------------------------------------------------------------- */
int fmm_probe_throughput(int kind, int iters, float* out, double* ops, void* stream);
int fmm_probe_blocks(void);

/* ---------------------------------------------------------------------------------------------
 * Parameter selector (no paper counterpart).  The paper picks the parameters by rule: p from the
 * tolerance through the error estimate of Section 3 (p ~ log TOL / log theta) and about 20 points
 * per leaf (end of Section 4).  The selector instead predicts the (levels, p) that meets a
 * tolerance fastest, with a small network trained on runs of the method itself:
 *
 *   features (64 binary32 per instance, fmm_selector_features): for levels l = 1..15 of a built
 *     tree, four statistics over the boxes of level l -- mean of log2(long side / root long side),
 *     standard deviation of log2(long side), mean and max of log2(long / short side) -- at
 *     [4(l-1) .. 4(l-1)+3] (zeros for missing levels); [60] log10 N, [61] log10 tol,
 *     [62] levels / 16, [63] 0.
 *   network: 64 -> 128 (ReLU) -> 128 (ReLU) -> 225 logits, softmax; class c means
 *     levels = 4 + c / 25, p = 8 + c % 25.  Parameters: one flat binary32 array of
 *     FMM_MLP_PARAMS values, row-major W1[128][64], b1[128], W2[128][128], b2[128],
 *     W3[225][128], b3[225] (y = W x + b).
 *   training: softmax cross-entropy averaged over the batch, Adam (beta1 0.9, beta2 0.999,
 *     eps 1e-8, bias-corrected), all on the GPU in binary32.
 * ------------------------------------------------------------------------------------------- */
#define FMM_MLP_IN 64
#define FMM_MLP_HIDDEN 128
#define FMM_MLP_OUT 225
#define FMM_MLP_PARAMS 53857
#define FMM_SEL_LMIN 4
#define FMM_SEL_LMAX 12
#define FMM_SEL_PMIN 8
#define FMM_SEL_PMAX 32
#define FMM_SEL_NP 25
#define FMM_FEAT_LOG10N 60
#define FMM_FEAT_LOG10TOL 61

typedef struct fmm_mlp_s* fmm_mlp;

/* Features of every instance of built tree t for tolerance 0 < tol < 1: features[n_inst][64]
 * (device, binary32).  The tree's device must be current. */
int fmm_selector_features(fmm_tree t, double tol, float* features, void* stream);

/* A network with room for batches of up to batch_max samples; parameters start at zero. */
int fmm_mlp_create(int batch_max, fmm_mlp* out);
void fmm_mlp_destroy(fmm_mlp m);

/* Copy parameters in (any memory cudaMemcpy can read; resets the Adam state) or out. */
int fmm_mlp_set_params(fmm_mlp m, const float* params, void* stream);
int fmm_mlp_get_params(fmm_mlp m, float* params, void* stream);

/* Class probabilities prob[B][225] of inputs X[B][64] (device). */
int fmm_mlp_forward(fmm_mlp m, const float* X, int B, float* prob, void* stream);

/* Gradient of the mean cross-entropy of labels[B] (device int32 classes) with respect to the
 * parameters, grad[FMM_MLP_PARAMS], and the mean loss loss[1] (device; either may be NULL).
 * A label outside [0, 225) makes the loss NaN. */
int fmm_mlp_gradients(fmm_mlp m, const float* X, const int32_t* labels, int B, float* grad, float* loss,
                      void* stream);

/* One Adam step with learning rate lr on the batch (X, labels); loss[1] (device, may be NULL)
 * receives the batch's mean loss before the step. */
int fmm_mlp_train_step(fmm_mlp m, const float* X, const int32_t* labels, int B, float lr, float* loss,
                       void* stream);

/* The selector's choice for B feature vectors (device): levels_p[B][2] = (levels, p) of the most
 * probable class among those whose levels lie in the window the training labels are drawn from,
 * Lc - 2 <= levels <= Lc + 1 with Lc = round(log4(N / 32)) rounded half up (= floor((b - 4) / 2),
 * b = floor(log2 N)), and have 4^levels <= N; N is read from the log10 N feature.  Where that
 * window is empty (very small N) every class with 4^levels <= N, and levels = 4, is allowed
 * (device int32). */
int fmm_select_params(fmm_mlp m, const float* features, int B, int32_t* levels_p, void* stream);

/* The complex field of Section 5's first experiment, G(z_i, z_j) = -q_j / (z_i - z_j):
 *     F_i = sum_{j != i} -q_j / (z_i - z_j)   (Re F = -dphi/dx, Im F = +dphi/dy of Eq. (1.1))
 * with the same tree, lists and expansions as fmm_evaluate: the far part is minus the derivative
 * of the local expansion, the near part the direct sum along the strong lists of the finest
 * level; coincident points contribute nothing.  fre[n], fim[n] (binary64, device) in INPUT order.
 * Modes and the tolerance rule as for fmm_evaluate; the binary32 near field keeps the
 * coordinates as float-float offsets from the leaf centres and handles leaves of up to 64
 * points (larger leaves take the binary64 path).  A leaf box of zero size (all its points
 * coincide, with at least two levels) has no scaled derivative: the device status then reports
 * FMM_ERR_DEGENERATE. */
int fmm_evaluate_field(fmm_tree t, fmm_lists l, const double* q, const fmm_params* prm, double* fre,
                       double* fim, void* stream);

/* The same field by direct summation in binary64 at m target input indices (int64, device). */
int fmm_direct_field(const double* x, const double* y, const double* q, int64_t n,
                     const int64_t* targets, int64_t m, double* fre, double* fim, void* stream);

/* Eq. (1.1) by direct summation in binary64 at m target input indices targets[m] (int64,
 * device) over all n sources; phi[m] (device).  Coincident distinct points contribute 0. */
int fmm_direct(const double* x, const double* y, const double* q, int64_t n,
               const int64_t* targets, int64_t m, double* phi, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Instrumentation (no paper counterpart): per-stage device times and a kernel launch counter,
 * used by the benchmark to report per-kernel rooflines.
 * ------------------------------------------------------------------------------------------- */
typedef enum {
    FMM_STAGE_TREE_SORT = 0,   /* keys, bounding box, the x and y radix sorts                 */
    FMM_STAGE_TREE_SPLIT = 1,  /* per-level stable partitions, split coordinates, rectangles  */
    FMM_STAGE_TREE_FINISH = 2, /* canonical order, box geometry, gathered coordinates         */
    FMM_STAGE_LISTS = 3,       /* strong/weak lists of all levels                              */
    FMM_STAGE_GATHER = 4,      /* strengths into canonical order                               */
    FMM_STAGE_P2M = 5,
    FMM_STAGE_M2M = 6,
    FMM_STAGE_M2L = 7,
    FMM_STAGE_L2L = 8,
    FMM_STAGE_LEAF = 9,        /* L2P, far and near joined in input order (the field: also its
                                  near sum, P2L and M2P)                                        */
    FMM_STAGE_NEAR = 10,       /* near-field direct sum of the potentials                     */
    FMM_STAGE_EXCHANGE = 11,   /* P2L and M2P of the role-exchange lists (potentials)         */
    FMM_STAGE_COUNT = 12
} fmm_stage;

/* Enable (on != 0) or disable recording of a CUDA event pair around every stage, on the stream
 * of the call that runs the stage.  Process-wide; meant for one device at a time. */
int fmm_profile_enable(int on);

/* Wait for the recorded events and add, per stage, the elapsed milliseconds to ms[stage] and
 * the number of recorded stage executions to count[stage] (host arrays of nstages entries, either
 * may be NULL); then forget the records.  Returns the number of records read or an error. */
int fmm_profile_read(double* ms_host, int64_t* count_host, int nstages);

/* Number of kernels the library has launched in this process so far. */
int64_t fmm_launch_count(void);

/* Wait for `stream` and return the first error recorded in the device status of the tree and
 * (if not NULL) the lists, then clear it. */
int fmm_sync_status(fmm_tree t, fmm_lists l, void* stream);

/* Message of the last error returned on the calling thread ("" if none). */
const char* fmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FMM_GB300_H */
