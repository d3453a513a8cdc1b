// Internal declarations shared by the translation units of libfmm_gb300.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fmm.h"

namespace fmm {

// ---- device status word bits (set by kernels with atomicOr, read by fmm_sync_status) ----
enum : int32_t { ST_NONFINITE = 1, ST_CAPACITY = 2, ST_TIMEOUT = 4, ST_ARG = 8, ST_DEGENERATE = 16 };

// ---- error reporting (thread-local message) ----
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define FMM_CUDA(call)                                             \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ::fmm::cuda_fail(e_, #call); \
    } while (0)

#define FMM_LAUNCH_CHECK(what)                                     \
    do {                                                           \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return ::fmm::cuda_fail(e_, what);  \
    } while (0)

// ---- instrumentation ----
void note_launch(int n = 1);                          // count kernels launched by the library
void prof_mark(int stage, bool begin, cudaStream_t s);  // CUDA event around a stage (if enabled)

struct StageScope {
    int stage;
    cudaStream_t s;
    StageScope(int st, cudaStream_t str) : stage(st), s(str) { prof_mark(stage, true, s); }
    ~StageScope() { prof_mark(stage, false, s); }
};

// Items per tile of the tree-build kernels (sorts and partitions): TREE_TPB threads x TREE_ITEMS.
constexpr int TREE_TPB = 256;
constexpr int TREE_ITEMS = 4;
constexpr int TREE_TILE = TREE_TPB * TREE_ITEMS;

// Weak-list entry naming the parent (level l - 1) of four weak siblings: index | PARENT_FLAG.
constexpr int32_t PARENT_FLAG = FMM_PARENT_FLAG;
// Exchange-list entry whose target is the larger leaf (M2P); without it the target takes P2L.
constexpr int32_t SWAP_M2P = FMM_SWAP_M2P;

// ---- level-order box numbering ----
__host__ __device__ inline int64_t level_base(int l) { return ((int64_t(1) << (2 * l)) - 1) / 3; }
__host__ __device__ inline int64_t level_size(int l) { return int64_t(1) << (2 * l); }

// Source box of a weak-list entry v of target box g (global ids within an instance): a box of
// g's level, or with PARENT_FLAG a box of the level above.
__device__ __forceinline__ int64_t weak_source(int64_t g, int32_t v)
{
    const int l = (63 - __clzll((unsigned long long)(3 * g + 1))) >> 1;
    return (v & PARENT_FLAG) ? level_base(l - 1) + (v & ~PARENT_FLAG) : level_base(l) + v;
}

// Target boxes of weak entries.  Entries are sorted by target (CSR over the boxes of an
// instance, woff[0] = woff[1] = 0); wrow holds the target of every eighth entry.  A reader of
// consecutive entries takes the target of its first entry from wrow (any entry: from the eighth
// before it) and steps through the offsets: while e >= woff[g + 1], g = g + 1.
__device__ __forceinline__ int64_t wtarget_start(const int32_t* __restrict__ wrow,
                                                 const int32_t* __restrict__ woff, int64_t e)
{
    int64_t g = wrow[e >> 3];
    while (e >= woff[g + 1]) g++;
    return g;
}

// The per-depth tables of ones_before are concatenated: depth d starts at 2^d - 1.
__host__ __device__ inline int64_t ones_before_offset(int depth) { return (int64_t(1) << depth) - 1; }

// Node offsets of depth d (2^d + 1 entries each) start at 2^d - 1 + d.
__host__ __device__ inline int64_t node_offset_base(int depth) { return (int64_t(1) << depth) - 1 + depth; }

// Descend the floor-left binary split tree of n positions by `depth` steps towards position
// `pos`; returns the index j of the node at that depth and its offset o and size m.  A node of
// size m has children of sizes floor(m/2) (left) and m - floor(m/2) (right); two steps make one
// quadtree level (x-halves, then y-halves), so the node index at depth 2l is the box index of
// level l.
__device__ __forceinline__ int64_t descend_pos(int64_t n, int depth, int64_t pos, int64_t& o,
                                               int64_t& m)
{
    int64_t j = 0;
    o = 0;
    m = n;
    for (int d = 0; d < depth; d++) {
        int64_t h = m >> 1;
        if (pos < o + h) {
            m = h;
            j = 2 * j;
        } else {
            o += h;
            m -= h;
            j = 2 * j + 1;
        }
    }
    return j;
}

// Offset and size of node j at `depth` (follow the bits of j from the most significant).
__device__ __forceinline__ void descend_node(int64_t n, int depth, int64_t j, int64_t& o, int64_t& m)
{
    o = 0;
    m = n;
    for (int d = depth - 1; d >= 0; d--) {
        int64_t h = m >> 1;
        if ((j >> d) & 1) {
            o += h;
            m -= h;
        } else {
            m = h;
        }
    }
}

}  // namespace fmm

// ---------------------------------------------------------------------------------------------
// Handles.  A tree handle holds a forest: one or more independent instances (point sets) whose
// arrays are concatenated.  Every kernel processes all instances of a launch, finds its instance
// from a block index and offsets its pointers with the instance's entry of the table below, so the
// kernel bodies index one instance's arrays exactly as for a single point set.
// ---------------------------------------------------------------------------------------------
namespace fmm {

struct Inst {
    int64_t p0, n;        // points [p0, p0 + n) of the concatenated point arrays
    int64_t b0, nbox;     // boxes [b0, b0 + nbox), level order inside the instance
    int64_t o0;           // CSR offsets of the lists: [o0, o0 + nbox + 1) (o0 = b0 + instance)
    int64_t t0, ntiles;   // tree-build tiles [t0, t0 + ntiles)
    int64_t ob0;          // ones-before tables: 2^(2L) - 1 entries
    int64_t no0;          // node-offset tables: 2^(2L+1) + 2L entries
    int64_t lb0;          // leaf offsets: 4^L + 1 entries
    int32_t L;
    int32_t maxleaf;      // points of the largest leaf (ceil(n / 4^L) on the median tree)
    int32_t lg;           // median tree: levels l < lg split by the global partition passes, the
                          // rest inside one block per box of level lg (lg == L: none)
};

// A box of at most TREE_LOCAL_CAP points finishes its median subtree inside one block.
constexpr int TREE_LOCAL_CAP = 4096;
constexpr int TREE_LOCAL_TPB = 512;

// Launch schedule over the instances of a forest.  A launch is a 1-D grid; block b works for
// instance inst[b] as the rank-th of the nb = span[inst].y blocks that instance received
// (span[inst].x is its first block).  Blocks are shared out in proportion to each instance's
// work, so small and large instances finish together.  A tree of one instance needs no tables:
// inst == nullptr means instance 0 owns the whole grid.
struct Sched {
    const int32_t* inst = nullptr;  // [blocks]
    const int2* span = nullptr;     // [n_inst]
};

struct Slot {
    int i, rank, nb;
};

__device__ __forceinline__ Slot slot_of(const Sched& m)
{
    if (m.inst == nullptr) return Slot{0, (int)blockIdx.x, (int)gridDim.x};
    const int i = __ldg(m.inst + blockIdx.x);
    const int2 sp = __ldg(m.span + i);
    return Slot{i, (int)blockIdx.x - sp.x, sp.y};
}

// Radix digit-count scans: digits handled by one block of an instance with `ntiles` tiles
// (digits x tiles <= 1024, so one block-wide scan covers them), or 1 from 1024 tiles on.
__host__ __device__ inline int rs_digits_per_block(int64_t ntiles)
{
    if (ntiles >= 1024) return 1;
    const int64_t g = 1024 / (ntiles < 1 ? 1 : ntiles);
    return (int)(g < 256 ? g : 256);
}

// Host side of a schedule: the device tables (owned by the tree) and the grid size.
struct SchedH {
    Sched d;
    int blocks = 0;
    void* mem = nullptr;
};

// An item of the upward (M2M) or downward (L2L) work queue: boxes [b0, b0 + nb) of one level of
// one instance (within-level indices; for the downward pass the parents whose children receive).
struct QItem {
    int32_t inst, level, b0, nb;
};
constexpr int QLEVELS = 64;  // per-instance stride of the queue counters

struct LInst {            // list storage of one instance
    int64_t w0, wcap;     // weak entries [w0, w0 + wcap) (w0 and wcap multiples of 8)
    int64_t s0, scap;     // strong entries [s0, s0 + scap)
    int64_t f0;           // candidate flags [f0, f0 + 16 scap + tile)
    int64_t c0;           // candidate tile counts
};

}  // namespace fmm

struct fmm_tree_s {
    int dev = 0;
    int n_inst = 0;
    int Lmax = 0;
    int64_t n = 0;          // total points
    int64_t nbox = 0;       // total boxes
    int64_t ntiles = 0;     // total tree-build tiles
    int64_t max_tiles = 0;  // largest per-instance tile count
    int64_t max_n = 0;      // largest instance
    int64_t nleaf = 0;      // total leaves
    int64_t n_ob = 0, n_no = 0;
    fmm::Inst* hinst = nullptr;   // host copy of the instance table [n_inst]
    fmm::Inst* dinst = nullptr;   // device copy
    bool own_hinst = true;

    // products of the build (device; concatenated over instances)
    double* rects = nullptr;     // [nbox][4] (x0, x1, y0, y1)
    double* centers = nullptr;   // [nbox][2]
    double* radii = nullptr;     // [nbox]
    float* rad32 = nullptr;      // [nbox] radii rounded to binary32
    float* cen_hi = nullptr;     // [nbox][2] float part of the centre
    float* cen_lo = nullptr;     // [nbox][2] float remainder (centre - hi)
    int32_t* perm = nullptr;     // [n] canonical order -> input index (local to the instance)
    int32_t* leaf_begin = nullptr;  // per instance [4^L + 1], local positions
    int32_t* leaf_of = nullptr;  // [n] leaf of each input index
    int32_t* cleaf = nullptr;    // [n] leaf of each canonical position
    double* xs = nullptr;        // [n] x in canonical order
    double* ys = nullptr;        // [n]
    float* dxf = nullptr;        // [n] x - leaf centre, binary32, canonical order
    float* dyf = nullptr;        // [n]

    // build scratch (device)
    uint64_t* keys = nullptr;    // [4][n] ping-pong keys for the x and y sorts
    int32_t* vals = nullptr;     // [4][n] ping-pong values
    uint32_t* rs_counts = nullptr;  // [2][256][ntiles] (per instance: [2][256][its tiles])
    uint32_t* rs_totals = nullptr;  // [n_inst][2][256]
    uint32_t* tilecnt = nullptr;    // [ntiles]
    uint8_t* hflag = nullptr;       // [2][n] per input index: x-half / y-half bit
    uint64_t* bbox_keys = nullptr;  // [n_inst][4] ordered keys of xmin, xmax, ymin, ymax
    int32_t* ones_before = nullptr;  // per instance, per depth 0 .. 2L-1: [2^depth]
    int32_t* node_off = nullptr;     // per instance, node offsets per depth 0 .. 2L: [2^depth + 1]
    int32_t* segs = nullptr;         // [4][n] box index carried by the items of X and Y
    int32_t* status = nullptr;       // device status word

    // expansion workspace (allocated by the first evaluate that needs it; PS = padded P)
    int ws_ps64 = 0, ws_ps32 = 0;
    void* Me = nullptr;   // binary64 multipoles [nbox][PS] (double2: re, im)
    void* Le = nullptr;   // binary64 locals     [nbox][PS]
    void* Mf = nullptr;   // binary32 multipoles [nbox][PS] (float2)
    void* Lf = nullptr;   // binary32 locals     [nbox][PS]
    void* pk64 = nullptr;   // [n] double4 (x, y, q, 0) in canonical order (binary64 path)
    void* pk32 = nullptr;   // [n] float4 (x - c_leaf, y - c_leaf, q, 0) (binary32 path)
    double* acc = nullptr;  // [n] binary64 potential accumulator in canonical order
    float* acc32 = nullptr; // [6n] binary32 accumulators: potential far hi, lo, near hi, lo; the field
                            // far re, im, near re hi, lo, im hi, lo (canonical order)
    void* pkf = nullptr;    // [n] float4 float-float offsets from the leaf centre (binary32 field)
    float* qf = nullptr;    // [n] strengths in canonical order (binary32 field)
    double* accf = nullptr; // [2n] binary64 field accumulator (re, im)
    float* Lf0lo = nullptr; // [nbox] low part of Re b_0 of the binary32 locals (float-float)
    void* pkff = nullptr;   // [n][2] float4: float-float offsets from the leaf centre and strength (split mode)
    void* mff = nullptr;    // [nbox][mff_ps] float4: float-float multipoles (split mode, role exchange)
    int mff_ps = 0;

    // launch tuning (set by fmm_autotune; 0 = defaults): total blocks of the M2L and near-field
    // launches, shared out over the instances in proportion to their work
    int tune_m2l_blocks = 0, tune_p2p_blocks = 0;
    int tune_m2l_chunk = 0;   // tensor-core M2L: consecutive weak entries per row (0 = default)
    int tune_m2l_stages = 0;  // tensor-core M2L: TMEM accumulator stages 1 or 2 (0 = by order)
    int tune_p2p_nt = 0;      // binary32 near field: targets per lane 2 or 4 (0 = default)
    int m2l_kind = 0;  // binary32 M2L: 0 = by order (tensor cores for 24 <= P <= 32), 1 = SIMT, 2 = tensor cores

    // launch schedules (device tables only for forests of more than one instance)
    fmm::SchedH s_tiles;   // one block per tree-build tile
    fmm::SchedH s_pts;     // blocks in proportion to the points
    fmm::SchedH s_rsscan;  // radix digit-count scans (groups of digits per block)
    fmm::SchedH s_p2m;     // the leaves, 4 per block
    fmm::SchedH s_m2l, s_p2p;
    fmm::SchedH s_local;   // boxes of level lg (instances with lg < L), one block each
    fmm::SchedH* s_split = nullptr;  // [Lmax] boxes of level l, 128 per block (levels l < L)
    fmm::SchedH* s_m2m = nullptr;    // [Lmax] boxes of level l, 4 per block (l < L)
    fmm::SchedH* s_l2l = nullptr;    // [Lmax] children of level l, 4 per block (l < L)
    fmm::SchedH* s_lists = nullptr;  // [Lmax + 1] candidate tiles of level l (l <= L)
    bool built = false;
    // uniform-grid mesh (the non-adaptive comparison of Section 5) in place of the median tree:
    // leaf offsets and largest leaves then come from the data; the balanced leaf offsets are kept
    // in lb_bal to restore them for the next median build
    bool uniform = false;
    // fmm_step: a second stream and its events, created on first use
    cudaStream_t side = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // lists done, points packed, near field done
    cudaEvent_t* ev_level = nullptr;  // [Lmax + 1]: geometry of a level complete
    int32_t* lb_bal = nullptr;
    // the upward and downward passes as persistent launches over work queues (expand.cu)
    void* qmem = nullptr;       // items up, items down, needs up, needs down, done counters, tickets
    int32_t nq_up = 0, nq_dn = 0;
    int64_t q_counter_bytes = 0;  // done counters and tickets, cleared before each pass
};

struct fmm_lists_s {
    fmm_tree tree = nullptr;
    int64_t wcap = 0, scap = 0;   // totals over instances
    fmm::LInst* hlinst = nullptr;
    fmm::LInst* dlinst = nullptr;
    int32_t* woff = nullptr;  // per instance [nbox + 1], local entry positions
    int32_t* soff = nullptr;
    int32_t* widx = nullptr;  // within-level index of the source box
    int32_t* wrow = nullptr;    // target box (local id) of weak entries 0, 8, 16, ...: [w0 / 8 + k]
    int32_t* rowtgt = nullptr;  // tensor-core M2L with rows of T % 8 != 0 entries: target of each row
    int32_t* sidx = nullptr;
    int32_t* stgt = nullptr;
    uint8_t* flags = nullptr;     // weak flag per candidate of the level being built
    uint32_t* tilecnt = nullptr;  // per-tile weak counts of the level being built
    int32_t* status = nullptr;
    double theta = 0.0;
    bool built = false;
    // Section 4's optional optimisations (mode bits): FMM_LISTS_PARENTS lets four weak siblings
    // become one entry naming their parent; tiledrop counts the siblings dropped per tile
    int mode = 0;
    uint32_t* tiledrop = nullptr;
    // finest-level role exchange (FMM_LISTS_EXCHANGE): per-tile counts and the exchange lists
    // (offsets in the layout of woff, entries in that of the strong lists)
    uint32_t* tileswap = nullptr;
    int32_t* xoff = nullptr;
    int32_t* xidx = nullptr;
    int32_t* xtgt = nullptr;  // target leaf (global id) of each exchange entry
    // general near-field kernel: work items per strong pair, their exclusive scan
    int32_t* p2p_items = nullptr;
    int32_t* p2p_pos = nullptr;
    uint32_t* p2p_tmp = nullptr;
    int32_t* p2p_zero = nullptr;
};

namespace fmm {

// sched.cu: build / free schedules.  blocks[i] = blocks of instance i (0 = none).
int sched_make(fmm_tree t, const int64_t* blocks, SchedH& out);
void sched_free(SchedH& h);
int sched_all(fmm_tree t);          // every schedule that depends on the instances only
int sched_tuned(fmm_tree t);        // the M2L and near-field schedules (depend on the tuning)
void sched_free_all(fmm_tree t);

// tree.cu
int tree_alloc(fmm_tree t, int n_inst, const int64_t* n, const int* levels);
void fill_instances(Inst* out, int n_inst, const int64_t* ns, const int* Ls);
void forest_totals(fmm_tree t);
int tree_tables_host(int64_t n, int L, int32_t* ones_before, int32_t* node_off, int32_t* leaf_begin);
// Once per device, outside any stream capture: kernel attributes the tree build needs.
int tree_kernel_setup();
// level_ready (may be null): events [Lmax + 1]; event l is recorded once the geometry (centres,
// radii) of levels 0 .. l is complete, so that the lists of those levels can be built meanwhile.
int tree_build(fmm_tree t, const double* x, const double* y, cudaStream_t s, cudaEvent_t* level_ready = nullptr);
int tree_build_uniform(fmm_tree t, const double* x, const double* y, const double* root_host, cudaStream_t s);

// lists.cu
// level_ready (may be null): wait for event l before building level l (see tree_build).
int lists_build(fmm_tree t, fmm_lists l, double theta, cudaStream_t s, const cudaEvent_t* level_ready = nullptr);
int64_t lists_flag_bytes(int64_t scap);
int64_t lists_tile_words(int64_t scap);
int lists_alloc(fmm_tree t, fmm_lists l, const int64_t* weak_capacity, const int64_t* strong_capacity);

// expand.cu
// Structural checks (fmm_validate) and list import (fmm_lists_import).
int validate(fmm_tree t, fmm_lists l, cudaStream_t s);
int lists_import(fmm_lists l, int i, const int32_t* woff, const int32_t* widx, const int32_t* soff,
                 const int32_t* sidx, cudaStream_t s);

// Two-stream step (fmm_step): the lists are built on `side` (lists_done when complete); the
// evaluation records `gathered` once the points are packed, and its binary32 near field runs on
// `side`, recording `near_done`.
struct StepSync {
    cudaStream_t side;
    cudaEvent_t lists_done, gathered, near_done;
};
int evaluate(fmm_tree t, fmm_lists l, const double* q, const fmm_params& prm, double* phi,
             cudaStream_t s, const StepSync* sync = nullptr);
int evaluate_field(fmm_tree t, fmm_lists l, const double* q, const fmm_params& prm, double* fre,
                   double* fim, cudaStream_t s);
int direct_field(const double* x, const double* y, const double* q, int64_t n, const int64_t* tgt,
                 int64_t m, double* fre, double* fim, cudaStream_t s);
int direct(const double* x, const double* y, const double* q, int64_t n, const int64_t* tgt,
           int64_t m, double* phi, cudaStream_t s);
int autotune(fmm_tree t, fmm_lists l, const double* q, const fmm_params& prm, double* phi,
             cudaStream_t s, int* m2l_blocks, int* p2p_blocks);
// Work queues of the upward and downward passes (built once per tree, from its instances).
int queues_make(fmm_tree t);
int queue_timeout_selftest(fmm_tree t, int64_t limit, cudaStream_t s);

// m2l_tc.cu: binary32 M2L on the tensor cores (Me, Le: [nbox][PS] float2)
bool m2l_tc_supported(int P);
int m2l_tc(fmm_tree t, fmm_lists l, int P, int PS, const void* Me, void* Le, cudaStream_t s);
int bounded_wait_selftest(int64_t limit, cudaStream_t s);

// scan.cu: exclusive scan of int32 counts with a base value read from device memory:
// out[i] = base[0] + sum_{j < i} in[j] for i = 0..m (out has m + 1 entries; out may alias
// nothing).  tmp needs scan_tmp_words(m) words.
int64_t scan_tmp_words(int64_t m);
int scan_with_base(const int32_t* in, int64_t m, const int32_t* base, int32_t* out, uint32_t* tmp,
                   cudaStream_t s);

}  // namespace fmm
