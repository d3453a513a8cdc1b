// Tree construction for callers that cannot allocate device memory.
//
// fmm_build_tree needs a tree handle, and creating one calls cudaMalloc.  Some callers cannot do
// that: code inside a host application whose own memory manager owns the device and must not be
// bypassed (an allocation outside it can fail or fragment the memory it manages), and
// latency-critical loops that cannot afford the device-wide synchronisation a cudaMalloc or
// cudaFree may cause.  fmm_build_tree_noalloc serves them: it runs
// the same build kernels, but every intermediate buffer lives in one file-scope device array of
// fixed size that each GPU loading the library keeps until the process exits.  The caller passes
// only inputs and outputs.
//
// Consequences of the shared array: calls on one device must not overlap in time (two streams,
// or two host threads, running the build at once would overwrite each other's intermediates),
// and the first call on a device looks up the array's device address, which should happen before
// any stream capture begins.  That address and the kernels' shared-memory opt-in are kept for the
// life of the process: after cudaDeviceReset the device's context is a new one, so a process that
// resets a device must not call this entry point on it again.
#include <mutex>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int64_t NA_MAX_N = FMM_NOALLOC_MAX_POINTS;
constexpr int NA_MAX_L = FMM_NOALLOC_MAX_LEVELS;
constexpr int64_t NA_MAX_NBOX = ((int64_t(1) << (2 * (NA_MAX_L + 1))) - 1) / 3;
constexpr int64_t NA_TILE = TREE_TILE;  // items per tile of the build kernels
constexpr int64_t NA_TILES = (NA_MAX_N + NA_TILE - 1) / NA_TILE;

constexpr int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

// Byte layout of the scratch array (every region 256-byte aligned).
struct Layout {
    int64_t inst, keys, vals, rs_counts, rs_totals, tilecnt, hflag, bbox, ones_before, node_off, segs,
        status, centers, radii, rad32, cen_hi, cen_lo, leaf_of, cleaf, xs, ys, dxf, dyf, total;
};

constexpr Layout make_layout()
{
    Layout L{};
    int64_t o = 0;
    L.inst = o;        o += align256(sizeof(Inst));
    L.keys = o;        o += align256(8 * 4 * NA_MAX_N);
    L.vals = o;        o += align256(4 * 4 * NA_MAX_N);
    L.rs_counts = o;   o += align256(4 * 2 * 256 * NA_TILES);
    L.rs_totals = o;   o += align256(4 * 2 * 256);
    L.tilecnt = o;     o += align256(4 * NA_TILES);
    L.hflag = o;       o += align256(2 * NA_MAX_N);
    L.bbox = o;        o += align256(8 * 4);
    L.ones_before = o; o += align256(4 * (int64_t(1) << (2 * NA_MAX_L)));
    L.node_off = o;    o += align256(4 * ((int64_t(1) << (2 * NA_MAX_L + 1)) + 2 * NA_MAX_L + 1));
    L.segs = o;        o += align256(4 * 4 * NA_MAX_N);
    L.status = o;      o += align256(4);
    L.centers = o;     o += align256(16 * NA_MAX_NBOX);
    L.radii = o;       o += align256(8 * NA_MAX_NBOX);
    L.rad32 = o;       o += align256(4 * NA_MAX_NBOX);
    L.cen_hi = o;      o += align256(8 * NA_MAX_NBOX);
    L.cen_lo = o;      o += align256(8 * NA_MAX_NBOX);
    L.leaf_of = o;     o += align256(4 * NA_MAX_N);
    L.cleaf = o;       o += align256(4 * NA_MAX_N);
    L.xs = o;          o += align256(8 * NA_MAX_N);
    L.ys = o;          o += align256(8 * NA_MAX_N);
    L.dxf = o;         o += align256(4 * NA_MAX_N);
    L.dyf = o;         o += align256(4 * NA_MAX_N);
    L.total = o;
    return L;
}

constexpr Layout kLayout = make_layout();

// The scratch array itself.  Host code must not use this name as an address: it only stands in
// for the device symbol, whose address each device reports through cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kLayout.total];

std::mutex g_na_mutex;
unsigned char* g_na_base[128] = {};

// Set-up, once per device, with that device current.
int scratch_base(unsigned char** out)
{
    int dev = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return fail(FMM_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_base[dev]) {  // the first call on this device (documented: before any capture)
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch of fmm_build_tree_noalloc)");
        const int rc = tree_kernel_setup();  // no tree handle was created on this path
        if (rc) return rc;
        g_na_base[dev] = (unsigned char*)p;
    }
    *out = g_na_base[dev];
    return 0;
}

// Per-depth "ones before" tables of the stable partitions, node offsets and leaf offsets; the
// same values the allocating path computes on the host.  One block; depths are independent.
__global__ void __launch_bounds__(1024) k_noalloc_tables(Inst S, Inst* inst, int64_t n, int L,
                                                         int32_t* ones_before, int32_t* node_off,
                                                         int32_t* leaf_begin)
{
    if (threadIdx.x == 0) *inst = S;  // the instance table of the build kernels
    for (int d = 0; d <= 2 * L; d++) {
        const int64_t nodes = int64_t(1) << d;
        int32_t* off = node_off + node_offset_base(d);
        for (int64_t j = threadIdx.x; j <= nodes; j += blockDim.x) {
            int64_t o = n, m = 0;
            if (j < nodes) descend_node(n, d, j, o, m);
            off[j] = (int32_t)o;
        }
    }
    __shared__ int64_t wt[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int d = 0; d < 2 * L; d++) {
        const int64_t nodes = int64_t(1) << d;
        int32_t* ob = ones_before + ones_before_offset(d);
        int64_t carry = 0;
        for (int64_t b0 = 0; b0 < nodes; b0 += blockDim.x) {
            const int64_t j = b0 + threadIdx.x;
            int64_t v = 0;
            if (j < nodes) {
                int64_t o, m;
                descend_node(n, d, j, o, m);
                v = m - m / 2;  // right-child size
            }
            int64_t x = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += y;
            }
            if (lane == 31) wt[w] = x;
            __syncthreads();
            if (w == 0) {
                int64_t s = lane < nw ? wt[lane] : 0;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int64_t y = __shfl_up_sync(0xffffffffu, s, off);
                    if (lane >= off) s += y;
                }
                if (lane < nw) wt[lane] = s;
            }
            __syncthreads();
            if (j < nodes) ob[j] = (int32_t)(carry + (w ? wt[w - 1] : 0) + x - v);
            carry += wt[nw - 1];
            __syncthreads();
        }
    }
    const int64_t nleaf = int64_t(1) << (2 * L);
    for (int64_t j = threadIdx.x; j <= nleaf; j += blockDim.x) {
        int64_t o = n, m = 0;
        if (j < nleaf) descend_node(n, 2 * L, j, o, m);
        leaf_begin[j] = (int32_t)o;
    }
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" int fmm_build_tree_noalloc(const double* x, const double* y, int64_t n, int levels,
                                      int32_t* perm, double* rects, int32_t* leaf_begin,
                                      int32_t* status, void* stream)
{
    if (!x || !y || !perm || !rects || !leaf_begin) return fail(FMM_ERR_ARG, "NULL argument");
    if (levels < 0 || levels > NA_MAX_L)
        return fail(FMM_ERR_ARG, "fmm_build_tree_noalloc: levels = %d outside [0, %d]", levels, NA_MAX_L);
    if (n < 1 || n > NA_MAX_N)
        return fail(FMM_ERR_ARG, "fmm_build_tree_noalloc: n = %lld outside [1, %lld] (the static scratch "
                    "holds at most %lld points; use fmm_build_tree for larger inputs)",
                    (long long)n, (long long)NA_MAX_N, (long long)NA_MAX_N);
    if (n < level_size(levels))
        return fail(FMM_ERR_LEVELS, "n = %lld < 4^%d: some leaf would be empty", (long long)n, levels);
    unsigned char* base = nullptr;
    int rc = scratch_base(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    fmm_tree_s t;  // a handle on the stack whose buffers are regions of the scratch array
    Inst hs;       // its one instance
    fill_instances(&hs, 1, &n, &levels);
    t.n_inst = 1;
    t.hinst = &hs;
    t.own_hinst = false;
    forest_totals(&t);
    // a single instance needs no schedule tables (only small host arrays of grid sizes)
    // the launch schedules hold small host arrays: freed on every way out of this function
    struct SchedGuard {
        fmm_tree_s* t;
        ~SchedGuard() { sched_free_all(t); }
    } guard{&t};
    rc = sched_all(&t);
    if (rc) return rc;
    const Layout& Lo = kLayout;
    t.dinst = (Inst*)(base + Lo.inst);
    t.keys = (uint64_t*)(base + Lo.keys);
    t.vals = (int32_t*)(base + Lo.vals);
    t.rs_counts = (uint32_t*)(base + Lo.rs_counts);
    t.rs_totals = (uint32_t*)(base + Lo.rs_totals);
    t.tilecnt = (uint32_t*)(base + Lo.tilecnt);
    t.hflag = (uint8_t*)(base + Lo.hflag);
    t.bbox_keys = (uint64_t*)(base + Lo.bbox);
    t.ones_before = (int32_t*)(base + Lo.ones_before);
    t.node_off = (int32_t*)(base + Lo.node_off);
    t.segs = (int32_t*)(base + Lo.segs);
    t.status = (int32_t*)(base + Lo.status);
    t.centers = (double*)(base + Lo.centers);
    t.radii = (double*)(base + Lo.radii);
    t.rad32 = (float*)(base + Lo.rad32);
    t.cen_hi = (float*)(base + Lo.cen_hi);
    t.cen_lo = (float*)(base + Lo.cen_lo);
    t.leaf_of = (int32_t*)(base + Lo.leaf_of);
    t.cleaf = (int32_t*)(base + Lo.cleaf);
    t.xs = (double*)(base + Lo.xs);
    t.ys = (double*)(base + Lo.ys);
    t.dxf = (float*)(base + Lo.dxf);
    t.dyf = (float*)(base + Lo.dyf);
    t.perm = perm;          // outputs go straight to the caller's arrays
    t.rects = rects;
    t.leaf_begin = leaf_begin;

    // the array keeps the previous call's contents: the status word must start at zero; every
    // other region is fully written before it is read
    FMM_CUDA(cudaMemsetAsync(t.status, 0, 4, s));
    k_noalloc_tables<<<1, 1024, 0, s>>>(hs, t.dinst, n, levels, t.ones_before, t.node_off, leaf_begin);
    note_launch();
    FMM_LAUNCH_CHECK("fmm_build_tree_noalloc: tables");
    rc = tree_build(&t, x, y, s);
    if (rc) return rc;
    if (status) FMM_CUDA(cudaMemcpyAsync(status, t.status, 4, cudaMemcpyDeviceToDevice, s));
    return FMM_OK;
}
