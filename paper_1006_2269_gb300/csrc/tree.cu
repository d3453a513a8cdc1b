// Tree construction on the GPU: Section 4 (median splits), Fig. 1.1, Fig. 4.1.
//
// Design.  The x- and y-orders of all points are obtained once, by two stable LSD radix sorts of
// order-preserving 64-bit keys (ties keep input order, i.e. are broken by input index).  The
// tree is then built level by level without any further sorting: a box of level l is a
// contiguous segment of both the x-ordered list X and the y-ordered list Y, and
//   * its x-split sends the first floor(n/2) entries of its X segment to the x-low half;
//   * a stable partition of its Y segment by that half bit leaves Y segmented by x-halves,
//     each still in y order, so the y-split of a half is again "the first floor(m/2)";
//   * a stable partition of each x-half of X by the y bit leaves X segmented by the children.
// Segment offsets follow from N alone (floor-left binary splits), so every kernel locates its
// segment by integer arithmetic, and the stable partitions are one global scan of the flag bits
// plus a per-segment correction taken from a host-computed table.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int TPB = TREE_TPB;        // threads per block of the tiled kernels
constexpr int ITEMS = TREE_ITEMS;    // items per thread
constexpr int TILE = TREE_TILE;      // items per tile
constexpr int WARPS = TPB / 32;
constexpr int WCHUNK = ITEMS * 32;   // contiguous items handled by one warp
constexpr int BINS = 256;            // radix digit of 8 bits

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Order-preserving key of a binary64 value (-0 and +0 share the key of +0).
__device__ __forceinline__ uint64_t order_key(double v)
{
    v = __dadd_rn(v, 0.0);  // -0 + 0 = +0 in round-to-nearest; every other value is unchanged
    uint64_t b = (uint64_t)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_value(uint64_t k)
{
    uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x <= 1024, multiple of 32).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_tmp, uint32_t& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < nw ? warp_tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_tmp[lane] = s;  // inclusive prefix of warp totals
    }
    __syncthreads();
    total = warp_tmp[nw - 1];
    uint32_t before = w ? warp_tmp[w - 1] : 0;
    __syncthreads();
    return before + x - v;
}

// ---- keys, bounding box and finiteness -------------------------------------------------------

__global__ void k_bbox_init(uint64_t* bbox)
{
    if (threadIdx.x == 0) {
        bbox[0] = ~0ull;
        bbox[1] = 0ull;
        bbox[2] = ~0ull;
        bbox[3] = 0ull;
    }
}

__global__ void k_make_keys(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                            uint64_t* __restrict__ kx, uint64_t* __restrict__ ky,
                            uint64_t* bbox, int32_t* status)
{
    uint64_t mnx = ~0ull, mxx = 0, mny = ~0ull, mxy = 0;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double a = x[i], b = y[i];
        bad |= !isfinite(a) || !isfinite(b);
        uint64_t ka = order_key(a), kb = order_key(b);
        kx[i] = ka;
        ky[i] = kb;
        mnx = min(mnx, ka);
        mxx = max(mxx, ka);
        mny = min(mny, kb);
        mxy = max(mxy, kb);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin((unsigned long long*)&bbox[0], (unsigned long long)mnx);
        atomicMax((unsigned long long*)&bbox[1], (unsigned long long)mxx);
        atomicMin((unsigned long long*)&bbox[2], (unsigned long long)mny);
        atomicMax((unsigned long long*)&bbox[3], (unsigned long long)mxy);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// The root rectangle is the tight bounding box.  The extreme keys are converted back to the
// exact coordinates (min/max involve no rounding).
__global__ void k_root_rect(const uint64_t* bbox, double* rects)
{
    if (threadIdx.x < 4) rects[threadIdx.x] = key_value(bbox[threadIdx.x]);
}

// ---- stable LSD radix sort (8-bit digits) ----------------------------------------------------
// blockIdx.y selects one of several independent sorts laid out `stride` elements apart.

template <typename K>
__global__ void __launch_bounds__(TPB) k_rs_hist(const K* __restrict__ keys, int64_t stride, int64_t n,
                                                 int shift, uint32_t* __restrict__ counts,
                                                 int64_t ntiles)
{
    __shared__ uint32_t h[BINS];
    keys += (int64_t)blockIdx.y * stride;
    counts += (int64_t)blockIdx.y * BINS * ntiles;
    for (int i = threadIdx.x; i < BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * TILE;
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < ITEMS; j++) {
        int64_t i = base + (int64_t)j * TPB + threadIdx.x;
        bool v = i < n;
        uint32_t d = v ? (uint32_t)((keys[i] >> shift) & (BINS - 1)) : 0xffffffffu;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        if (v && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < BINS; i += blockDim.x) counts[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

// One block per (digit, sort): exclusive scan of that digit's per-tile counts, in place.
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* counts, int64_t ntiles, uint32_t* totals)
{
    __shared__ uint32_t wt[32];
    uint32_t* c = counts + ((int64_t)blockIdx.y * BINS + blockIdx.x) * ntiles;
    uint32_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        uint32_t v = i < ntiles ? c[i] : 0;
        uint32_t tot;
        uint32_t e = block_excl_scan(v, wt, tot);
        if (i < ntiles) c[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.y * BINS + blockIdx.x] = carry;
}

// Stable scatter.  Each warp owns WCHUNK consecutive items and walks them in order, ranking
// equal digits with match_any; warps are then ordered by a per-digit scan, tiles by k_rs_scan,
// digits by the scan of the totals.  With FIRST the values are the item indices.
template <typename K, bool FIRST>
__global__ void __launch_bounds__(TPB) k_rs_scatter(const K* __restrict__ kin, const int32_t* __restrict__ vin,
                                                    K* __restrict__ kout, int32_t* __restrict__ vout,
                                                    int64_t stride, int64_t n, int shift,
                                                    const uint32_t* __restrict__ counts,
                                                    const uint32_t* __restrict__ totals, int64_t ntiles)
{
    __shared__ uint32_t dbase[BINS];
    __shared__ uint32_t wcnt[WARPS][BINS];
    __shared__ uint32_t wt[32];
    const int64_t so = (int64_t)blockIdx.y * stride;
    kin += so;
    kout += so;
    vout += so;
    if (!FIRST) vin += so;
    counts += (int64_t)blockIdx.y * BINS * ntiles;
    totals += blockIdx.y * BINS;
    {
        uint32_t tot;
        uint32_t e = block_excl_scan(threadIdx.x < BINS ? totals[threadIdx.x] : 0, wt, tot);
        if (threadIdx.x < BINS) dbase[threadIdx.x] = e;
    }
    for (int i = threadIdx.x; i < WARPS * BINS; i += TPB) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)w * WCHUNK;
    K k[ITEMS];
    int32_t val[ITEMS];
    uint32_t r[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        int64_t i = base + j * 32 + lane;
        bool valid = i < n;
        k[j] = valid ? kin[i] : K(0);
        val[j] = valid ? (FIRST ? (int32_t)i : vin[i]) : 0;
        uint32_t d = valid ? (uint32_t)((k[j] >> shift) & (BINS - 1)) : (uint32_t)BINS;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t cur = valid ? wcnt[w][d] : 0;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = cur + __popc(peers);
        __syncwarp();
        r[j] = cur + __popc(peers & lt);
    }
    __syncthreads();
    if (threadIdx.x < BINS) {
        uint32_t run = 0;
        for (int ww = 0; ww < WARPS; ww++) {
            uint32_t c = wcnt[ww][threadIdx.x];
            wcnt[ww][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        int64_t i = base + j * 32 + lane;
        if (i < n) {
            uint32_t d = (uint32_t)((k[j] >> shift) & (BINS - 1));
            int64_t pos = (int64_t)dbase[d] + counts[(int64_t)d * ntiles + blockIdx.x] + wcnt[w][d] + r[j];
            kout[pos] = k[j];
            vout[pos] = val[j];
        }
    }
}

// Sorts `nsorts` independent arrays of n keys laid out `stride` apart; buffer A holds the input
// keys, buffer B = A + n (same for values).  Returns the index (0 = A, 1 = B) holding the result.
template <typename K>
int radix_sort(K* keys, int32_t* vals, int64_t stride, int nsorts, int64_t n, int bits,
               uint32_t* counts, uint32_t* totals, int64_t ntiles, cudaStream_t s)
{
    int cur = 0;
    dim3 grid((unsigned)ntiles, (unsigned)nsorts);
    for (int shift = 0; shift < bits; shift += 8) {
        K* kin = keys + (cur ? n : 0);
        K* kout = keys + (cur ? 0 : n);
        int32_t* vin = vals + (cur ? n : 0);
        int32_t* vout = vals + (cur ? 0 : n);
        k_rs_hist<K><<<grid, TPB, 0, s>>>(kin, stride, n, shift, counts, ntiles); note_launch();
        k_rs_scan<<<dim3(BINS, nsorts), 1024, 0, s>>>(counts, ntiles, totals); note_launch();
        if (shift == 0)
            k_rs_scatter<K, true><<<grid, TPB, 0, s>>>(kin, nullptr, kout, vout, stride, n, shift,
                                                       counts, totals, ntiles);
        else
            k_rs_scatter<K, false><<<grid, TPB, 0, s>>>(kin, vin, kout, vout, stride, n, shift,
                                                        counts, totals, ntiles);
        note_launch();
        cur ^= 1;
    }
    return cur;
}

// ---- stable partitions inside segments ---------------------------------------------------------

__global__ void __launch_bounds__(TPB) k_part_count(const int32_t* __restrict__ in,
                                                    const uint8_t* __restrict__ flag, int64_t n,
                                                    uint32_t* __restrict__ tilecnt)
{
    __shared__ uint32_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * TILE;
    uint32_t c = 0;
    for (int j = 0; j < ITEMS; j++) {
        int64_t i = base + (int64_t)j * TPB + threadIdx.x;
        if (i < n) c += flag[in[i]];
    }
    uint32_t tot;
    block_excl_scan(c, wt, tot);
    if (threadIdx.x == 0) tilecnt[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(uint32_t* a, int64_t m)
{
    __shared__ uint32_t wt[32];
    uint32_t carry = 0;
    for (int64_t b = 0; b < m; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        uint32_t v = i < m ? a[i] : 0;
        uint32_t tot;
        uint32_t e = block_excl_scan(v, wt, tot);
        if (i < m) a[i] = carry + e;
        carry += tot;
    }
}

// Stable partition inside segments.  Items carry the index of their level-l box (seg, a node at
// depth 2l of the floor-left split tree whose offsets are tabulated in node_off).
//   xmode = 0 (the y-ordered list): segments are the boxes themselves, flag = x-half bit; an item
//       lands in its x-half (depth 2l+1), where the y order makes its y-half bit "position in the
//       upper half"; out_seg receives the level-(l+1) box, flagout the y-half bit.
//   xmode = 1 (the x-ordered list): segments are the x-halves (depth 2l+1, the half follows from
//       the position), flag = y-half bit; out_seg receives the level-(l+1) box, flagout the
//       x-half bit of the next level.
// Zeros keep their order and come first.  A segment of size m holds m - floor(m/2) ones, ob[j]
// counts the ones of all segments before segment j at that depth, tileoff[] is the exclusive scan
// of the ones per tile.
__global__ void __launch_bounds__(TPB) k_part_scatter(const int32_t* __restrict__ in,
                                                      const int32_t* __restrict__ in_seg,
                                                      int32_t* __restrict__ out,
                                                      int32_t* __restrict__ out_seg,
                                                      const uint8_t* __restrict__ flag,
                                                      uint8_t* __restrict__ flagout, int32_t n, int l,
                                                      int xmode, const int32_t* __restrict__ node_off,
                                                      const int32_t* __restrict__ ones_before,
                                                      const uint32_t* __restrict__ tileoff,
                                                      int32_t* status)
{
    __shared__ uint32_t wtot[WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int32_t base = (int32_t)blockIdx.x * TILE + w * WCHUNK;
    const int32_t* offD = node_off + node_offset_base(2 * l);
    const int32_t* ob = ones_before + ones_before_offset(2 * l + xmode);
    int32_t id[ITEMS];
    uint32_t pre[ITEMS];
    uint32_t fl = 0, run = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const int32_t i = base + j * 32 + lane;
        const bool valid = i < n;
        id[j] = valid ? in[i] : 0;
        const uint32_t f = valid ? flag[id[j]] : 0;
        fl |= f << j;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        pre[j] = run + __popc(bal & lt);
        run += __popc(bal);
    }
    if (lane == 0) wtot[w] = run;
    __syncthreads();
    uint32_t woff = tileoff[blockIdx.x];
    for (int ww = 0; ww < w; ww++) woff += wtot[ww];
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const int32_t i = base + j * 32 + lane;
        if (i >= n) continue;
        const int32_t G = (int32_t)(woff + pre[j]);
        const int32_t seg = in_seg[i];
        int32_t o = offD[seg], m = offD[seg + 1] - o;
        int32_t seg1 = seg;
        if (xmode) {  // the x-half of the box
            const int32_t h = m >> 1;
            const int32_t bit = i >= o + h;
            seg1 = 2 * seg + bit;
            if (bit) {
                o += h;
                m -= h;
            } else {
                m = h;
            }
        }
        const int32_t ones = G - ob[seg1];
        const int32_t h = m >> 1;
        const int32_t f = (fl >> j) & 1;
        const int32_t np = f ? (o + h + ones) : (i - ones);
        if (np < o || np >= o + m) {  // cannot happen for consistent tables; never write out of range
            atomicOr(status, ST_ARG);
            continue;
        }
        const int32_t o2 = f ? o + h : o, m2 = f ? m - h : h;
        const int32_t seg2 = 2 * seg1 + f;
        const int32_t bit2 = np >= o2 + (m2 >> 1);
        out[np] = id[j];
        out_seg[np] = xmode ? seg2 : 2 * seg2 + bit2;
        flagout[id[j]] = (uint8_t)bit2;
    }
}

// Level-0 x-split: the upper half of the x order has the bit set.
__global__ void k_init_hx(const int32_t* __restrict__ X, int32_t n, uint8_t* __restrict__ hx)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        hx[X[i]] = (i >= (n >> 1)) ? 1 : 0;
}

__device__ __forceinline__ double midpoint(double a, double b) { return __dmul_rn(0.5, __dadd_rn(a, b)); }

// Split coordinates of the boxes of level l and the rectangles of their children.  X is the
// x-ordered list segmented by the boxes of level l, Yn the y-ordered list segmented by their
// x-halves.
__global__ void k_split_rects(const int32_t* __restrict__ X, const int32_t* __restrict__ Yn,
                              const double* __restrict__ x, const double* __restrict__ y,
                              const int32_t* __restrict__ node_off, int l, double* __restrict__ rects)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= level_size(l)) return;
    const int32_t* offD = node_off + node_offset_base(2 * l);
    const int64_t o = offD[b], m = offD[b + 1] - o;
    int64_t mx = m >> 1;
    double xs = midpoint(x[X[o + mx - 1]], x[X[o + mx]]);
    int64_t ho[2] = {o, o + mx}, hm[2] = {mx, m - mx};
    double ys[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        int64_t my = hm[h] >> 1;
        ys[h] = midpoint(y[Yn[ho[h] + my - 1]], y[Yn[ho[h] + my]]);
    }
    const double* pr = rects + 4 * (level_base(l) + b);
    double px0 = pr[0], px1 = pr[1], py0 = pr[2], py1 = pr[3];
    double* cr = rects + 4 * (level_base(l + 1) + 4 * b);
    cr[0] = px0; cr[1] = xs;  cr[2] = py0;   cr[3] = ys[0];
    cr[4] = px0; cr[5] = xs;  cr[6] = ys[0]; cr[7] = py1;
    cr[8] = xs;  cr[9] = px1; cr[10] = py0;  cr[11] = ys[1];
    cr[12] = xs; cr[13] = px1; cr[14] = ys[1]; cr[15] = py1;
}

// After the last level every item of X carries its leaf.
__global__ void k_leaf_of(const int32_t* __restrict__ X, const int32_t* __restrict__ XS, int32_t n,
                          uint32_t* __restrict__ leaf_of)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        leaf_of[X[i]] = (uint32_t)XS[i];
}

// Centre (rectangle midpoint) and radius (half diagonal) of every box, with the same sequence of
// correctly rounded binary64 operations as the criterion's reference; plus a float-float copy
// of the centre for the binary32 path.
__global__ void k_geometry(const double* __restrict__ rects, int64_t nbox, double* __restrict__ cen,
                           double* __restrict__ rad, float* __restrict__ rad32, float* __restrict__ chi,
                           float* __restrict__ clo)
{
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nbox) return;
    const double* r = rects + 4 * g;
    double w = __dsub_rn(r[1], r[0]), h = __dsub_rn(r[3], r[2]);
    double cx = midpoint(r[0], r[1]), cy = midpoint(r[2], r[3]);
    cen[2 * g] = cx;
    cen[2 * g + 1] = cy;
    const double rg = __dmul_rn(0.5, __dsqrt_rn(__dadd_rn(__dmul_rn(w, w), __dmul_rn(h, h))));
    rad[g] = rg;
    rad32[g] = __double2float_rn(rg);
    float hx = __double2float_rn(cx), hy = __double2float_rn(cy);
    chi[2 * g] = hx;
    chi[2 * g + 1] = hy;
    clo[2 * g] = __double2float_rn(__dsub_rn(cx, (double)hx));
    clo[2 * g + 1] = __double2float_rn(__dsub_rn(cy, (double)hy));
}

// Coordinates in canonical order, and their binary32 offsets from the leaf centre.
__global__ void k_gather_points(const int32_t* __restrict__ perm, const uint32_t* __restrict__ leaf_of,
                                const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                                int L, const double* __restrict__ cen, double* __restrict__ xs,
                                double* __restrict__ ys, float* __restrict__ dxf, float* __restrict__ dyf,
                                int32_t* __restrict__ cleaf)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t id = perm[i];
        cleaf[i] = (int32_t)leaf_of[id];
        int64_t g = level_base(L) + leaf_of[id];
        double a = x[id], b = y[id];
        xs[i] = a;
        ys[i] = b;
        dxf[i] = __double2float_rn(__dsub_rn(a, cen[2 * g]));
        dyf[i] = __double2float_rn(__dsub_rn(b, cen[2 * g + 1]));
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

}  // namespace

// Host side: sizes are fixed by (n, L) alone, so all tables are computed here once.
int tree_alloc(fmm_tree t)
{
    const int64_t n = t->n;
    const int L = t->L;
    t->nbox = level_base(L + 1);
    t->nleaf = level_size(L);
    t->ntiles = (n + TILE - 1) / TILE;

    // floor-left split sizes per depth; ones-before tables for depths 0 .. 2L-1; node offsets for
    // depths 0 .. 2L; leaf offsets
    std::vector<int64_t> sizes{n}, next;
    std::vector<int32_t> ob_all, off_all;
    for (int d = 0; d <= 2 * L; d++) {
        int64_t o = 0;
        for (int64_t m : sizes) {
            off_all.push_back((int32_t)o);
            o += m;
        }
        off_all.push_back((int32_t)o);
        if (d == 2 * L) break;
        int64_t acc = 0;
        for (int64_t m : sizes) {
            ob_all.push_back((int32_t)acc);
            acc += m - m / 2;
        }
        next.clear();
        for (int64_t m : sizes) {
            next.push_back(m / 2);
            next.push_back(m - m / 2);
        }
        sizes.swap(next);
    }
    std::vector<int32_t> lb(sizes.size() + 1);
    lb[0] = 0;
    for (size_t i = 0; i < sizes.size(); i++) lb[i + 1] = lb[i] + (int32_t)sizes[i];

    auto A = [&](void** p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) return fail(FMM_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        return 0;
    };
    int rc = 0;
    const size_t nb = (size_t)t->nbox, nn = (size_t)n;
    if ((rc = A((void**)&t->rects, 32 * nb))) return rc;
    if ((rc = A((void**)&t->centers, 16 * nb))) return rc;
    if ((rc = A((void**)&t->radii, 8 * nb))) return rc;
    if ((rc = A((void**)&t->rad32, 4 * nb))) return rc;
    if ((rc = A((void**)&t->cen_hi, 8 * nb))) return rc;
    if ((rc = A((void**)&t->cen_lo, 8 * nb))) return rc;
    if ((rc = A((void**)&t->perm, 4 * nn))) return rc;
    if ((rc = A((void**)&t->leaf_begin, 4 * lb.size()))) return rc;
    if ((rc = A((void**)&t->leaf_of, 4 * nn))) return rc;
    if ((rc = A((void**)&t->cleaf, 4 * nn))) return rc;
    if ((rc = A((void**)&t->xs, 8 * nn))) return rc;
    if ((rc = A((void**)&t->ys, 8 * nn))) return rc;
    if ((rc = A((void**)&t->dxf, 4 * nn))) return rc;
    if ((rc = A((void**)&t->dyf, 4 * nn))) return rc;
    if ((rc = A((void**)&t->keys, 8 * 4 * nn))) return rc;
    if ((rc = A((void**)&t->vals, 4 * 4 * nn))) return rc;
    if ((rc = A((void**)&t->rs_counts, 4 * 2 * BINS * (size_t)t->ntiles))) return rc;
    if ((rc = A((void**)&t->rs_totals, 4 * 2 * BINS))) return rc;
    if ((rc = A((void**)&t->tilecnt, 4 * (size_t)t->ntiles))) return rc;
    if ((rc = A((void**)&t->hflag, 2 * nn))) return rc;
    if ((rc = A((void**)&t->bbox_keys, 32))) return rc;
    if ((rc = A((void**)&t->ones_before, 4 * ob_all.size()))) return rc;
    if ((rc = A((void**)&t->node_off, 4 * off_all.size()))) return rc;
    if ((rc = A((void**)&t->segs, 4 * 4 * nn))) return rc;
    if ((rc = A((void**)&t->status, 4))) return rc;
    FMM_CUDA(cudaMemcpy(t->leaf_begin, lb.data(), 4 * lb.size(), cudaMemcpyHostToDevice));
    if (!ob_all.empty())
        FMM_CUDA(cudaMemcpy(t->ones_before, ob_all.data(), 4 * ob_all.size(), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemcpy(t->node_off, off_all.data(), 4 * off_all.size(), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemset(t->status, 0, 4));
    return 0;
}

int tree_build(fmm_tree t, const double* x, const double* y, cudaStream_t s)
{
    const int64_t n = t->n;
    const int L = t->L;
    const int64_t nt = t->ntiles;
    uint64_t* kx = t->keys;          // x sort: buffers [0, n) and [n, 2n)
    int32_t* vals = t->vals;         // x sort values [0, 2n); y sort values [2n, 4n)
    uint8_t* hx = t->hflag;
    uint8_t* hy = t->hflag + n;
    int32_t *X, *Xo, *Y, *Yo;
    int32_t* Xfinal_seg = nullptr;

    {
        StageScope scope(FMM_STAGE_TREE_SORT, s);
        k_bbox_init<<<1, 32, 0, s>>>(t->bbox_keys); note_launch();
        k_make_keys<<<grid_for(n, 256), 256, 0, s>>>(x, y, n, kx, kx + 2 * n, t->bbox_keys, t->status); note_launch();
        k_root_rect<<<1, 32, 0, s>>>(t->bbox_keys, t->rects); note_launch();
        FMM_LAUNCH_CHECK("tree: keys");
        // x order and y order of all points, ties by input index (two sorts in one launch sequence)
        int cur = radix_sort<uint64_t>(kx, vals, 2 * n, 2, n, 64, t->rs_counts, t->rs_totals, nt, s);
        FMM_LAUNCH_CHECK("tree: radix sort");
        X = vals + (cur ? n : 0);
        Xo = vals + (cur ? 0 : n);
        Y = vals + 2 * n + (cur ? n : 0);
        Yo = vals + 2 * n + (cur ? 0 : n);
    }

    {
        StageScope scope(FMM_STAGE_TREE_SPLIT, s);
        // box index carried by every item of X and Y (all in the root at level 0)
        int32_t *XS = t->segs, *XSo = t->segs + n, *YS = t->segs + 2 * n, *YSo = t->segs + 3 * n;
        FMM_CUDA(cudaMemsetAsync(XS, 0, 4 * n, s));
        FMM_CUDA(cudaMemsetAsync(YS, 0, 4 * n, s));
        const int32_t n32 = (int32_t)n;
        k_init_hx<<<grid_for(n, 256), 256, 0, s>>>(X, n32, hx); note_launch();
        for (int l = 0; l < L; l++) {
            // Y: stable partition of each box by its x-half bit; records the y-half bit
            k_part_count<<<(unsigned)nt, TPB, 0, s>>>(Y, hx, n, t->tilecnt); note_launch();
            k_scan_tiles<<<1, 1024, 0, s>>>(t->tilecnt, nt); note_launch();
            k_part_scatter<<<(unsigned)nt, TPB, 0, s>>>(Y, YS, Yo, YSo, hx, hy, n32, l, 0, t->node_off,
                                                        t->ones_before, t->tilecnt, t->status); note_launch();
            std::swap(Y, Yo);
            std::swap(YS, YSo);
            // split coordinates and child rectangles of level l
            int64_t nb = level_size(l);
            k_split_rects<<<(unsigned)((nb + 127) / 128), 128, 0, s>>>(X, Y, x, y, t->node_off, l, t->rects); note_launch();
            // X: stable partition of each x-half by the y-half bit; records the next x-half bit
            k_part_count<<<(unsigned)nt, TPB, 0, s>>>(X, hy, n, t->tilecnt); note_launch();
            k_scan_tiles<<<1, 1024, 0, s>>>(t->tilecnt, nt); note_launch();
            k_part_scatter<<<(unsigned)nt, TPB, 0, s>>>(X, XS, Xo, XSo, hy, hx, n32, l, 1, t->node_off,
                                                        t->ones_before, t->tilecnt, t->status); note_launch();
            std::swap(X, Xo);
            std::swap(XS, XSo);
            FMM_LAUNCH_CHECK("tree: level split");
        }
        Xfinal_seg = XS;
    }

    {
        StageScope scope(FMM_STAGE_TREE_FINISH, s);
        // canonical order: stable sort of the input indices by leaf (inside a leaf: input order)
        uint32_t* leaf_of = (uint32_t*)t->leaf_of;
        k_leaf_of<<<grid_for(n, 256), 256, 0, s>>>(X, Xfinal_seg, (int32_t)n, leaf_of); note_launch();
        uint32_t* k32 = (uint32_t*)t->keys;  // reuse the key buffers: [0, n) and [n, 2n)
        int32_t* v32 = t->vals + 2 * n;      // value buffers [2n, 4n)
        int bits = std::max(8, 2 * L);  // with L = 0 all keys are 0 and the order stays the input order
        FMM_CUDA(cudaMemcpyAsync(k32, leaf_of, 4 * n, cudaMemcpyDeviceToDevice, s));
        int c2 = radix_sort<uint32_t>(k32, v32, 0, 1, n, bits, t->rs_counts, t->rs_totals, nt, s);
        FMM_CUDA(cudaMemcpyAsync(t->perm, v32 + (c2 ? n : 0), 4 * n, cudaMemcpyDeviceToDevice, s));

        int64_t nb = t->nbox;
        k_geometry<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(t->rects, nb, t->centers, t->radii,
                                                                t->rad32, t->cen_hi, t->cen_lo); note_launch();
        k_gather_points<<<grid_for(n, 256), 256, 0, s>>>(t->perm, leaf_of, x, y, n, L, t->centers,
                                                         t->xs, t->ys, t->dxf, t->dyf, t->cleaf); note_launch();
        FMM_LAUNCH_CHECK("tree: canonical order");
    }
    t->built = true;
    return 0;
}

}  // namespace fmm
