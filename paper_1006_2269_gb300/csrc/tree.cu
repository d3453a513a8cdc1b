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
// Segment offsets follow from N alone (floor-left binary splits) and are tabulated once, items
// carry the index of their box, and the stable partitions are one scan of the flag bits per tile
// plus a per-segment correction from a table.
//
// A tree handle may hold many independent instances (a forest); every kernel covers all of them
// in one launch: a schedule tells each block its instance (and its rank among that instance's
// blocks), and the kernel offsets its pointers by the instance's entry of the instance table, so
// the bodies below index one point set.
#include <algorithm>
#include <new>
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

// Lanes of the warp holding the same 9-bit value d (digits 0..255, 256 for "no item"): one
// ballot per bit, each lane keeping the lanes that agree with it on that bit.
__device__ __forceinline__ unsigned match_digit(uint32_t d)
{
    unsigned m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 9; b++) {
        const bool bit = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bal : ~bal;
    }
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

__global__ void k_bbox_init(int n_inst, uint64_t* bbox)
{
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
        bbox[4 * i + 0] = ~0ull;
        bbox[4 * i + 1] = 0ull;
        bbox[4 * i + 2] = ~0ull;
        bbox[4 * i + 3] = 0ull;
    }
}

// schedule: points
__global__ void k_make_keys(Sched sc, const Inst* __restrict__ I, const double* __restrict__ x,
                            const double* __restrict__ y, int64_t ntot, uint64_t* __restrict__ kx,
                            uint64_t* bbox, int32_t* status)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    x += S.p0;
    y += S.p0;
    uint64_t* ky = kx + 2 * ntot + S.p0;  // the y keys live 2 ntot further
    kx += S.p0;
    bbox += 4 * z.i;
    uint64_t mnx = ~0ull, mxx = 0, mny = ~0ull, mxy = 0;
    bool bad = false;
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x) {
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
    // then across the block, so that only one thread per block touches the four shared words
    __shared__ uint64_t red[4][32];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = mnx;
        red[1][w] = mxx;
        red[2][w] = mny;
        red[3][w] = mxy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; k++) {
            mnx = min(mnx, red[0][k]);
            mxx = max(mxx, red[1][k]);
            mny = min(mny, red[2][k]);
            mxy = max(mxy, red[3][k]);
        }
        atomicMin((unsigned long long*)&bbox[0], (unsigned long long)mnx);
        atomicMax((unsigned long long*)&bbox[1], (unsigned long long)mxx);
        atomicMin((unsigned long long*)&bbox[2], (unsigned long long)mny);
        atomicMax((unsigned long long*)&bbox[3], (unsigned long long)mxy);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// The root rectangle is the tight bounding box.  The extreme keys are converted back to the
// exact coordinates (min/max involve no rounding).
__global__ void k_root_rect(const Inst* __restrict__ I, int n_inst, const uint64_t* bbox, double* rects)
{
    for (int i = threadIdx.x; i < 4 * n_inst; i += blockDim.x)
        rects[4 * I[i / 4].b0 + (i % 4)] = key_value(bbox[i]);
}

// ---- stable LSD radix sort (8-bit digits) ----------------------------------------------------
// grid (tile schedule, sorts): one block per tile of an instance.  Sort `srt` of an instance uses
// keys[srt * stride + p0 ...] and counts [2][256][its tiles] at 2 * 256 * t0.

template <typename K>
__global__ void __launch_bounds__(TPB) k_rs_hist(Sched sc, const Inst* __restrict__ I, const K* __restrict__ keys,
                                                 int64_t stride, int shift, uint32_t* __restrict__ counts)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const int64_t tile = z.rank;
    __shared__ uint32_t h[BINS];
    keys += (int64_t)blockIdx.y * stride + S.p0;
    counts += 2 * BINS * S.t0 + (int64_t)blockIdx.y * BINS * S.ntiles;
    for (int i = threadIdx.x; i < BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = tile * TILE;
    const int lane = threadIdx.x & 31;
    // one shared-memory atomic per item; a warp whose items all share one digit (the high digits
    // of clustered or narrow-range coordinates) adds its 32 at once instead of 32 colliding ones
    uint32_t d[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const int64_t i = base + (int64_t)j * TPB + threadIdx.x;
        d[j] = i < S.n ? (uint32_t)((keys[i] >> shift) & (BINS - 1)) : 0xffffffffu;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const uint32_t d0 = __shfl_sync(0xffffffffu, d[j], 0);
        if (__all_sync(0xffffffffu, d[j] == d0)) {
            if (lane == 0 && d0 != 0xffffffffu) atomicAdd(&h[d0], 32u);
        } else if (d[j] != 0xffffffffu) {
            atomicAdd(&h[d[j]], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < BINS; i += blockDim.x) counts[(int64_t)i * S.ntiles + tile] = h[i];
}

// grid (digit-group schedule, sorts): exclusive scans of the per-tile counts of every digit, in
// place, and each digit's total.  A block takes G = rs_digits_per_block(ntiles) consecutive
// digits of one instance: below 1024 tiles their counts (G x ntiles <= 1024 values) go through one
// block-wide scan whose segments are the digits; from 1024 tiles on G = 1 and the digit is scanned
// in chunks of 1024.
__global__ void __launch_bounds__(1024) k_rs_scan(Sched sc, const Inst* __restrict__ I, uint32_t* counts,
                                                  uint32_t* totals)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    __shared__ uint32_t wt[32];
    __shared__ uint32_t ex[1024];
    const int64_t nt = S.ntiles;
    const int G = rs_digits_per_block(nt);
    const int d0 = z.rank * G;
    if (d0 >= BINS) return;
    uint32_t* c = counts + 2 * BINS * S.t0 + (int64_t)blockIdx.y * BINS * nt + (int64_t)d0 * nt;
    uint32_t* tot = totals + (2 * (int64_t)z.i + blockIdx.y) * BINS + d0;
    if (nt >= 1024) {
        uint32_t carry = 0;
        for (int64_t b = 0; b < nt; b += blockDim.x) {
            const int64_t i = b + threadIdx.x;
            const uint32_t v = i < nt ? c[i] : 0;
            uint32_t t;
            const uint32_t e = block_excl_scan(v, wt, t);
            if (i < nt) c[i] = carry + e;
            carry += t;
        }
        if (threadIdx.x == 0) tot[0] = carry;
        return;
    }
    const int nd = min(G, BINS - d0);
    const int64_t len = (int64_t)nd * nt;
    const int k = threadIdx.x;
    const uint32_t v = k < len ? c[k] : 0;
    uint32_t t;
    const uint32_t e = block_excl_scan(v, wt, t);
    ex[k] = e;
    __syncthreads();
    if (k < len) {
        const int k0 = k - (int)(k % nt);
        c[k] = e - ex[k0];
        if (k % nt == nt - 1) tot[k / nt] = e + v - ex[k0];
    }
}

// Stable scatter.  Each warp owns WCHUNK consecutive items and walks them in order, ranking
// equal digits with match_any; warps are then ordered by a per-digit scan, tiles by k_rs_scan,
// digits by the scan of the totals.  With FIRST the values are the item indices.
template <typename K, bool FIRST>
__global__ void __launch_bounds__(TPB) k_rs_scatter(Sched sc, const Inst* __restrict__ I, const K* __restrict__ kin,
                                                    const int32_t* __restrict__ vin,
                                                    K* __restrict__ kout, int32_t* __restrict__ vout,
                                                    int64_t stride, int shift,
                                                    const uint32_t* __restrict__ counts,
                                                    const uint32_t* __restrict__ totals)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const int64_t tile = z.rank;
    __shared__ uint32_t dbase[BINS];
    __shared__ uint32_t wcnt[WARPS][BINS];
    __shared__ uint32_t wt[32];
    const int64_t so = (int64_t)blockIdx.y * stride + S.p0;
    kin += so;
    kout += so;
    vout += so;
    if (!FIRST) vin += so;
    counts += 2 * BINS * S.t0 + (int64_t)blockIdx.y * BINS * S.ntiles;
    totals += (2 * (int64_t)z.i + blockIdx.y) * BINS;
    const int64_t n = S.n;
    {
        // digit d of this tile starts at (digits below d over all tiles) + (digit d in the tiles
        // before this one)
        uint32_t tot;
        uint32_t e = block_excl_scan(threadIdx.x < BINS ? totals[threadIdx.x] : 0, wt, tot);
        if (threadIdx.x < BINS) dbase[threadIdx.x] = e + counts[(int64_t)threadIdx.x * S.ntiles + tile];
    }
    for (int i = threadIdx.x; i < WARPS * BINS; i += TPB) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t base = tile * TILE + (int64_t)w * WCHUNK;
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
        unsigned peers = match_digit(d);
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
            int64_t pos = (int64_t)dbase[d] + wcnt[w][d] + r[j];
            kout[pos] = k[j];
            vout[pos] = val[j];
        }
    }
}

// Sorts `nsorts` arrays per instance; buffer A holds the input keys, buffer B = A + ntot (same for
// values).  Returns the index (0 = A, 1 = B) holding the result.
template <typename K>
int radix_sort(fmm_tree t, K* keys, int32_t* vals, int64_t stride, int nsorts, int bits,
               cudaStream_t s)
{
    int cur = 0;
    const int64_t ntot = t->n;
    const dim3 grid((unsigned)t->s_tiles.blocks, (unsigned)nsorts);
    const dim3 gscan((unsigned)t->s_rsscan.blocks, (unsigned)nsorts);
    const Sched st = t->s_tiles.d;
    for (int shift = 0; shift < bits; shift += 8) {
        K* kin = keys + (cur ? ntot : 0);
        K* kout = keys + (cur ? 0 : ntot);
        int32_t* vin = vals + (cur ? ntot : 0);
        int32_t* vout = vals + (cur ? 0 : ntot);
        k_rs_hist<K><<<grid, TPB, 0, s>>>(st, t->dinst, kin, stride, shift, t->rs_counts); note_launch();
        k_rs_scan<<<gscan, 1024, 0, s>>>(t->s_rsscan.d, t->dinst, t->rs_counts, t->rs_totals); note_launch();
        if (shift == 0)
            k_rs_scatter<K, true><<<grid, TPB, 0, s>>>(st, t->dinst, kin, nullptr, kout, vout, stride, shift,
                                                       t->rs_counts, t->rs_totals);
        else
            k_rs_scatter<K, false><<<grid, TPB, 0, s>>>(st, t->dinst, kin, vin, kout, vout, stride, shift,
                                                        t->rs_counts, t->rs_totals);
        note_launch();
        cur ^= 1;
    }
    return cur;
}

// ---- stable partitions inside segments ---------------------------------------------------------

// tile schedule
__global__ void __launch_bounds__(TPB) k_part_count(Sched sc, const Inst* __restrict__ I, int l,
                                                    const int32_t* __restrict__ in,
                                                    const uint8_t* __restrict__ flag,
                                                    uint32_t* __restrict__ tilecnt)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    if (l >= S.lg) return;
    in += S.p0;
    flag += S.p0;
    __shared__ uint32_t wt[32];
    const int64_t base = (int64_t)z.rank * TILE;
    uint32_t c = 0;
    for (int j = 0; j < ITEMS; j++) {
        int64_t i = base + (int64_t)j * TPB + threadIdx.x;
        if (i < S.n) c += flag[in[i]];
    }
    uint32_t tot;
    block_excl_scan(c, wt, tot);
    if (threadIdx.x == 0) tilecnt[S.t0 + z.rank] = tot;
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
// counts the ones of all segments before segment j at that depth, tilecnt[] the ones of every
// tile (each block adds up those before its own).  An instance with fewer than l + 1 levels is finished: its items are
// copied through unchanged so that the next level finds them in the output buffer; so is one
// whose remaining levels are split inside blocks (l >= lg).
// tile schedule
__global__ void __launch_bounds__(TPB) k_part_scatter(Sched sc, const Inst* __restrict__ I, int l, int xmode,
                                                      const int32_t* __restrict__ in,
                                                      const int32_t* __restrict__ in_seg,
                                                      int32_t* __restrict__ out,
                                                      int32_t* __restrict__ out_seg,
                                                      const uint8_t* __restrict__ flag,
                                                      uint8_t* __restrict__ flagout,
                                                      const int32_t* __restrict__ node_off,
                                                      const int32_t* __restrict__ ones_before,
                                                      const uint32_t* __restrict__ tilecnt,
                                                      int32_t* status)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const int32_t tile = z.rank;
    in += S.p0;
    in_seg += S.p0;
    out += S.p0;
    out_seg += S.p0;
    const int32_t n = (int32_t)S.n;
    if (l >= S.lg) {
        for (int j = 0; j < ITEMS; j++) {
            const int32_t i = tile * TILE + j * TPB + threadIdx.x;
            if (i < n) {
                out[i] = in[i];
                out_seg[i] = in_seg[i];
            }
        }
        return;
    }
    flag += S.p0;
    flagout += S.p0;
    __shared__ uint32_t wtot[WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int32_t base = tile * TILE + w * WCHUNK;
    const int32_t* offD = node_off + S.no0 + node_offset_base(2 * l);
    const int32_t* ob = ones_before + S.ob0 + ones_before_offset(2 * l + xmode);
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
    // ones before this tile: the sum of the earlier tiles' counts (no separate scan launch)
    __shared__ uint32_t wpart[WARPS];
    {
        uint32_t part = 0;
        for (int32_t k = threadIdx.x; k < tile; k += TPB) part += tilecnt[S.t0 + k];
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) wpart[w] = part;
    }
    __syncthreads();
    uint32_t woff = 0;
    for (int ww = 0; ww < WARPS; ww++) woff += wpart[ww];
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

// Level-0 x-split: the upper half of the x order has the bit set.  schedule: points
__global__ void k_init_hx(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ X, uint8_t* __restrict__ hx)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    X += S.p0;
    hx += S.p0;
    const int32_t n = (int32_t)S.n;
    for (int32_t i = z.rank * blockDim.x + threadIdx.x; i < n; i += z.nb * blockDim.x)
        hx[X[i]] = (i >= (n >> 1)) ? 1 : 0;
}

__device__ __forceinline__ double midpoint(double a, double b) { return __dmul_rn(0.5, __dadd_rn(a, b)); }

// The four children of box b of level l from its x-split xs and the y-splits of its halves.
__device__ __forceinline__ void child_rects(double* __restrict__ rects, int l, int64_t b, double xs,
                                            const double ys[2])
{
    const double* pr = rects + 4 * (level_base(l) + b);
    double px0 = pr[0], px1 = pr[1], py0 = pr[2], py1 = pr[3];
    double* cr = rects + 4 * (level_base(l + 1) + 4 * b);
    cr[0] = px0; cr[1] = xs;  cr[2] = py0;   cr[3] = ys[0];
    cr[4] = px0; cr[5] = xs;  cr[6] = ys[0]; cr[7] = py1;
    cr[8] = xs;  cr[9] = px1; cr[10] = py0;  cr[11] = ys[1];
    cr[12] = xs; cr[13] = px1; cr[14] = ys[1]; cr[15] = py1;
}

__device__ __forceinline__ void split_one(int64_t b, int l, const int32_t* __restrict__ X,
                                          const int32_t* __restrict__ Yn, const double* __restrict__ x,
                                          const double* __restrict__ y, const int32_t* __restrict__ offD,
                                          double* __restrict__ rects)
{
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
    child_rects(rects, l, b, xs, ys);
}

// Split coordinates of the boxes of level l and the rectangles of their children.  X is the
// x-ordered list segmented by the boxes of level l, Yn the y-ordered list segmented by their
// x-halves.  schedule: boxes of level l, one thread each
__global__ void k_split_rects(Sched sc, const Inst* __restrict__ I, int l, const int32_t* __restrict__ X,
                              const int32_t* __restrict__ Yn, const double* __restrict__ x,
                              const double* __restrict__ y, const int32_t* __restrict__ node_off,
                              double* __restrict__ rects)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    if (l >= S.lg) return;
    X += S.p0;
    Yn += S.p0;
    x += S.p0;
    y += S.p0;
    rects += 4 * S.b0;
    const int32_t* offD = node_off + S.no0 + node_offset_base(2 * l);
    for (int64_t b = (int64_t)z.rank * blockDim.x + threadIdx.x; b < level_size(l); b += (int64_t)z.nb * blockDim.x)
        split_one(b, l, X, Yn, x, y, offD, rects);
}

// After the last level every item of X carries its leaf.  schedule: points
__global__ void k_leaf_of(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ X,
                          const int32_t* __restrict__ XS, uint32_t* __restrict__ leaf_of)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    X += S.p0;
    XS += S.p0;
    leaf_of += S.p0;
    const int32_t n = (int32_t)S.n;
    for (int32_t i = z.rank * blockDim.x + threadIdx.x; i < n; i += z.nb * blockDim.x)
        leaf_of[X[i]] = (uint32_t)XS[i];
}

// Centre (rectangle midpoint) and radius (half diagonal) of every box, with the same sequence of
// correctly rounded binary64 operations as the criterion's reference; plus a float-float copy
// of the centre and a binary32 radius for the binary32 path.  One thread per box of the forest.
__device__ __forceinline__ void geometry_one(int64_t g, const double* __restrict__ rects, double* __restrict__ cen,
                                             double* __restrict__ rad, float* __restrict__ rad32,
                                             float* __restrict__ chi, float* __restrict__ clo)
{
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

__global__ void k_geometry(const double* __restrict__ rects, int64_t nbox, double* __restrict__ cen,
                           double* __restrict__ rad, float* __restrict__ rad32, float* __restrict__ chi,
                           float* __restrict__ clo)
{
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nbox) return;
    geometry_one(g, rects, cen, rad, rad32, chi, clo);
}

// The roots of every instance; one block.
__global__ void k_geometry_roots(const Inst* __restrict__ I, int n_inst, const double* __restrict__ rects,
                                 double* __restrict__ cen, double* __restrict__ rad, float* __restrict__ rad32,
                                 float* __restrict__ chi, float* __restrict__ clo)
{
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) geometry_one(I[i].b0, rects, cen, rad, rad32, chi, clo);
}

// The same for the boxes of level l of every instance split by the global passes (as soon as
// their rectangles exist; the block-local split does the levels below lg itself).
// schedule: boxes of level l - 1 (128 per block), four children each
__global__ void k_geometry_level(Sched sc, const Inst* __restrict__ I, int l, const double* __restrict__ rects,
                                 double* __restrict__ cen, double* __restrict__ rad, float* __restrict__ rad32,
                                 float* __restrict__ chi, float* __restrict__ clo)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    if (l > S.lg) return;
    const int64_t nb = level_size(l);
    for (int64_t b = (int64_t)z.rank * blockDim.x + threadIdx.x; b < nb; b += (int64_t)z.nb * blockDim.x)
        geometry_one(S.b0 + level_base(l) + b, rects, cen, rad, rad32, chi, clo);
}

// ---- the lowest levels inside one block per box -------------------------------------------------
// A box of level lg with m <= TREE_LOCAL_CAP points finishes its subtree (levels lg .. L-1) in
// shared memory, with the three steps of every global level: a stable partition of the y-ordered
// list by the x-half bit, the split coordinates and child rectangles, a stable partition of the
// x-ordered list by the y-half bit.  Points are renamed by their position in the box's x order at
// level lg (local ids < m), and segment indices are local to the subtree: node j at relative
// depth d is node (b << d) + j of the instance, whose offset and ones-before count come from the
// same tables as in the global passes.  Both therefore build the same tree.  At the end the
// x-ordered list (segmented by leaves) and each item's leaf go back to X and XS in place.
struct LocalSmem {
    int32_t gid[TREE_LOCAL_CAP];                            // local id -> point of the instance
    uint16_t xl[2][TREE_LOCAL_CAP], yl[2][TREE_LOCAL_CAP];  // x and y orders of local ids
    uint16_t xs[2][TREE_LOCAL_CAP], ys[2][TREE_LOCAL_CAP];  // their segment indices
    uint8_t hx[TREE_LOCAL_CAP], hy[TREE_LOCAL_CAP];         // half bits, by local id
    uint32_t wt[32];
};
static_assert(TREE_LOCAL_CAP <= 65536, "local ids and segment indices are 16-bit");
constexpr int LOC_IPT = TREE_LOCAL_CAP / TREE_LOCAL_TPB;  // consecutive items of one thread
static_assert(LOC_IPT * TREE_LOCAL_TPB == TREE_LOCAL_CAP && LOC_IPT <= 32, "items per thread");

// One stable partition of the block's lists, as k_part_scatter does it for a whole instance.
// offA: node offsets of the level-l boxes of the subtree (depth 2l, from its first node); obA:
// ones-before counts of the segments at depth 2l + XMODE (from the subtree's first node); o: the
// box's offset in the instance.
template <int XMODE>
__device__ __forceinline__ void local_partition(LocalSmem& sm, int cur, int32_t m, int32_t nseg,
                                                const int32_t* __restrict__ offA, const int32_t* __restrict__ obA,
                                                int32_t o, int32_t* status)
{
    const uint16_t* lst = XMODE ? sm.xl[cur] : sm.yl[cur];
    const uint16_t* seg = XMODE ? sm.xs[cur] : sm.ys[cur];
    uint16_t* lo = XMODE ? sm.xl[cur ^ 1] : sm.yl[cur ^ 1];
    uint16_t* so = XMODE ? sm.xs[cur ^ 1] : sm.ys[cur ^ 1];
    const uint8_t* fin = XMODE ? sm.hy : sm.hx;
    uint8_t* fout = XMODE ? sm.hx : sm.hy;
    const int32_t k0 = (int32_t)threadIdx.x * LOC_IPT;
    uint32_t fl = 0, c = 0;
#pragma unroll
    for (int j = 0; j < LOC_IPT; j++) {
        const int32_t k = k0 + j;
        const uint32_t f = k < m ? fin[lst[k]] : 0u;
        fl |= f << j;
        c += f;
    }
    uint32_t tot;
    uint32_t G = block_excl_scan(c, sm.wt, tot);  // ones before this thread's first item
    const int32_t ob0 = obA[0];
#pragma unroll
    for (int j = 0; j < LOC_IPT; j++) {
        const int32_t k = k0 + j;
        if (k >= m) break;
        const uint32_t f = (fl >> j) & 1u;
        const int32_t sg = seg[k];
        if (sg >= nseg) {  // cannot happen: segment indices of depth 2l are < 4^(l - lg)
            atomicOr(status, ST_ARG);
            G += f;
            continue;
        }
        int32_t os = offA[sg] - o, ms = offA[sg + 1] - offA[sg];
        int32_t s1 = sg;
        if (XMODE) {  // the x-half of the box
            const int32_t h = ms >> 1;
            const int32_t bit = k >= os + h;
            s1 = 2 * sg + bit;
            if (bit) {
                os += h;
                ms -= h;
            } else {
                ms = h;
            }
        }
        const int32_t ones = (int32_t)G - (obA[s1] - ob0);
        G += f;
        const int32_t h = ms >> 1;
        const int32_t np = f ? (os + h + ones) : (k - ones);
        if (np < os || np >= os + ms || np < 0 || np >= m) {  // cannot happen for consistent tables
            atomicOr(status, ST_ARG);
            continue;
        }
        const int32_t o2 = f ? os + h : os, m2 = f ? ms - h : h;
        const int32_t s2 = 2 * s1 + (int32_t)f;
        const int32_t bit2 = np >= o2 + (m2 >> 1);
        const uint16_t id = lst[k];
        lo[np] = id;
        so[np] = (uint16_t)(XMODE ? s2 : 2 * s2 + bit2);
        fout[id] = (uint8_t)bit2;
    }
    __syncthreads();
}

// schedule: boxes of level lg of the instances with lg < L, one block each (TREE_LOCAL_TPB
// threads, sizeof(LocalSmem) bytes of dynamic shared memory).  scratch: n int32 per instance
// (the local id of every point of the box).  geo != 0: also the geometry of the new boxes.
__global__ void __launch_bounds__(TREE_LOCAL_TPB, 2)
k_split_local(Sched sc, const Inst* __restrict__ I, int32_t* __restrict__ X, int32_t* __restrict__ XS,
              const int32_t* __restrict__ Y, const double* __restrict__ x, const double* __restrict__ y,
              const int32_t* __restrict__ node_off, const int32_t* __restrict__ ones_before,
              int32_t* __restrict__ scratch, double* __restrict__ rects, double* __restrict__ cen,
              double* __restrict__ rad, float* __restrict__ rad32, float* __restrict__ chi,
              float* __restrict__ clo, int geo, int32_t* status)
{
    extern __shared__ __align__(16) unsigned char local_smem[];
    LocalSmem& sm = *reinterpret_cast<LocalSmem*>(local_smem);
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const int lg = S.lg, L = S.L;
    if (lg >= L) return;
    const int64_t b = z.rank;  // the box of level lg
    X += S.p0;
    XS += S.p0;
    Y += S.p0;
    x += S.p0;
    y += S.p0;
    scratch += S.p0;
    const int32_t* nodes = node_off + S.no0;
    const int32_t* obt = ones_before + S.ob0;
    const int32_t o = nodes[node_offset_base(2 * lg) + b];
    const int32_t m = nodes[node_offset_base(2 * lg) + b + 1] - o;
    if (m < 0 || m > TREE_LOCAL_CAP || o < 0 || (int64_t)o + m > S.n) {  // block-uniform
        if (threadIdx.x == 0) atomicOr(status, ST_CAPACITY);
        return;
    }
    const int32_t n = (int32_t)S.n;
    for (int32_t k = threadIdx.x; k < m; k += blockDim.x) {
        const int32_t g = X[o + k];
        const bool ok = g >= 0 && g < n;
        if (!ok) atomicOr(status, ST_ARG);
        sm.gid[k] = ok ? g : 0;
        sm.xl[0][k] = (uint16_t)k;
        sm.xs[0][k] = 0;
        sm.ys[0][k] = 0;
        sm.hx[k] = (uint8_t)(k >= (m >> 1));  // x-half of the box: the upper half of its x order
        if (ok) scratch[g] = k;
    }
    __syncthreads();
    for (int32_t k = threadIdx.x; k < m; k += blockDim.x) {
        const int32_t g = Y[o + k];
        int32_t v = (g >= 0 && g < n) ? scratch[g] : -1;
        if (v < 0 || v >= m) {
            atomicOr(status, ST_ARG);
            v = 0;
        }
        sm.yl[0][k] = (uint16_t)v;
    }
    __syncthreads();
    double* R = rects + 4 * S.b0;
    int cx = 0, cy = 0;
    for (int l = lg; l < L; l++) {
        const int r = l - lg;
        const int32_t* offA = nodes + node_offset_base(2 * l) + (b << (2 * r));
        // Y: stable partition of every box by its x-half bit; records the y-half bits
        const int32_t nseg = (int32_t)level_size(r);
        local_partition<0>(sm, cy, m, nseg, offA, obt + ones_before_offset(2 * l) + (b << (2 * r)), o, status);
        cy ^= 1;
        // split coordinates and child rectangles of the subtree's boxes of level l
        for (int32_t sb = threadIdx.x; sb < nseg; sb += blockDim.x) {
            const int32_t os = offA[sb] - o, mb = offA[sb + 1] - offA[sb];
            if (mb < 4 || os < 0 || os + mb > m) {  // every box above the leaves holds >= 4 points
                atomicOr(status, ST_ARG);
                continue;
            }
            const int32_t mx = mb >> 1;
            const double xsp = midpoint(x[sm.gid[sm.xl[cx][os + mx - 1]]], x[sm.gid[sm.xl[cx][os + mx]]]);
            const int32_t ho[2] = {os, os + mx}, hm[2] = {mx, mb - mx};
            double ysp[2];
#pragma unroll
            for (int hh = 0; hh < 2; hh++) {
                const int32_t my = hm[hh] >> 1;
                ysp[hh] = midpoint(y[sm.gid[sm.yl[cy][ho[hh] + my - 1]]], y[sm.gid[sm.yl[cy][ho[hh] + my]]]);
            }
            const int64_t B = (b << (2 * r)) + sb;
            child_rects(R, l, B, xsp, ysp);
            if (geo)
                for (int c = 0; c < 4; c++)
                    geometry_one(S.b0 + level_base(l + 1) + 4 * B + c, rects, cen, rad, rad32, chi, clo);
        }
        // X: stable partition of each x-half by the y-half bit; records the next x-half bits
        local_partition<1>(sm, cx, m, nseg, offA, obt + ones_before_offset(2 * l + 1) + (b << (2 * r + 1)), o, status);
        cx ^= 1;
    }
    const int64_t leaf0 = b << (2 * (L - lg));
    for (int32_t k = threadIdx.x; k < m; k += blockDim.x) {
        X[o + k] = sm.gid[sm.xl[cx][k]];
        XS[o + k] = (int32_t)(leaf0 + sm.xs[cx][k]);
    }
}

// Canonical order inside small leaves.  After the last split the x-ordered list X holds every
// leaf as one contiguous run (XS: its leaf), at the leaf's offsets; the canonical order sorts each
// run by input index.  With at most LEAF_RANK_MAX points per leaf, each point's place in its run
// is the number of smaller indices in it (indices are distinct), found by one pass over the run.
// schedule: points
constexpr int LEAF_RANK_MAX = 64;
__global__ void k_leaf_rank(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ X,
                            const int32_t* __restrict__ XS, const int32_t* __restrict__ leaf_begin,
                            int32_t* __restrict__ perm, int32_t* __restrict__ cleaf, int32_t* status)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    X += S.p0;
    XS += S.p0;
    perm += S.p0;
    cleaf += S.p0;
    const int32_t* lb = leaf_begin + S.lb0;
    const int32_t n = (int32_t)S.n, nleaf = (int32_t)level_size(S.L);
    for (int32_t i = z.rank * blockDim.x + threadIdx.x; i < n; i += z.nb * blockDim.x) {
        const int32_t lf = XS[i];
        const int32_t a = (lf >= 0 && lf < nleaf) ? lb[lf] : 0, e = (lf >= 0 && lf < nleaf) ? lb[lf + 1] : 0;
        if (i < a || i >= e || e - a > LEAF_RANK_MAX) {  // not a run of this leaf: the tree is broken
            atomicOr(status, ST_ARG);
            continue;
        }
        const int32_t v = X[i];
        int32_t r = 0;
        for (int32_t k = a; k < e; k++) r += X[k] < v;
        perm[a + r] = v;
        cleaf[a + r] = lf;
    }
}

// Coordinates in canonical order, and their binary32 offsets from the leaf centre.  The leaf of
// each position comes from leaf_of (by input index) or, when leaf_of is null, from cleaf, which
// k_leaf_rank has filled already.
// schedule: points
__global__ void k_gather_points(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ perm,
                                const uint32_t* __restrict__ leaf_of, const double* __restrict__ x,
                                const double* __restrict__ y, const double* __restrict__ cen,
                                double* __restrict__ xs, double* __restrict__ ys,
                                float* __restrict__ dxf, float* __restrict__ dyf,
                                int32_t* __restrict__ cleaf)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    perm += S.p0;
    leaf_of += S.p0;
    x += S.p0;
    y += S.p0;
    xs += S.p0;
    ys += S.p0;
    dxf += S.p0;
    dyf += S.p0;
    cleaf += S.p0;
    cen += 2 * S.b0;
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x) {
        int32_t id = perm[i];
        int32_t lf;
        if (leaf_of) {
            lf = (int32_t)leaf_of[id];
            cleaf[i] = lf;
        } else {
            lf = cleaf[i];
        }
        int64_t g = level_base(S.L) + lf;
        double a = x[id], b = y[id];
        xs[i] = a;
        ys[i] = b;
        dxf[i] = __double2float_rn(__dsub_rn(a, cen[2 * g]));
        dyf[i] = __double2float_rn(__dsub_rn(b, cen[2 * g + 1]));
    }
}

// ---- uniform-grid mesh (the non-adaptive comparison of Section 5) -----------------------------
// Root: the square [x0, x0 + side] x [y0, y0 + side] on the bounding box's lower-left corner with
// its longer side; every box splits into four equal quadrants (children numbered as in the median
// tree).  Cell (ix, iy) of level l spans x0 + side * (ix / 2^l) .. x0 + side * ((ix + 1) / 2^l);
// a point's leaf has ix = floor(((x - x0) / side) * 2^L) clamped to [0, 2^L - 1] (iy likewise, all
// 0 when side = 0).  Binary64 with explicit rounding, so the mesh is the same bit for bit on any
// machine that rounds to nearest.

// The root square: given (x0, y0, side) when root.z >= 0, else the bounding square.
__device__ __forceinline__ double root_square(const uint64_t* bb, double3 root, double& x0, double& y0)
{
    if (root.z >= 0.0) {
        x0 = root.x;
        y0 = root.y;
        return root.z;
    }
    x0 = key_value(bb[0]);
    y0 = key_value(bb[2]);
    const double sx = __dsub_rn(key_value(bb[1]), x0), sy = __dsub_rn(key_value(bb[3]), y0);
    return sx > sy ? sx : sy;
}

// leaf of every point (input order); schedule: points
__global__ void k_uniform_cells(Sched sc, const Inst* __restrict__ I, const double* __restrict__ x,
                                const double* __restrict__ y, const uint64_t* __restrict__ bbox, double3 root,
                                uint32_t* __restrict__ leaf_of)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    x += S.p0;
    y += S.p0;
    leaf_of += S.p0;
    double x0, y0;
    const double side = root_square(bbox + 4 * z.i, root, x0, y0);
    const int L = S.L;
    const int64_t m = int64_t(1) << L;
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x) {
        int64_t ix = 0, iy = 0;
        if (side > 0.0) {
            ix = (int64_t)floor(__dmul_rn(__ddiv_rn(__dsub_rn(x[i], x0), side), (double)m));
            iy = (int64_t)floor(__dmul_rn(__ddiv_rn(__dsub_rn(y[i], y0), side), (double)m));
            ix = min(max(ix, (int64_t)0), m - 1);
            iy = min(max(iy, (int64_t)0), m - 1);
        }
        uint32_t id = 0;
        for (int j = L - 1; j >= 0; j--) id = 4 * id + 2 * ((ix >> j) & 1) + ((iy >> j) & 1);
        leaf_of[i] = id;
    }
}

// leaf offsets from the leaf ids in canonical (sorted) order: lb[c] = first position whose id is
// >= c; schedule: points (position j = n closes the table)
__global__ void k_uniform_lb(Sched sc, const Inst* __restrict__ I, const uint32_t* __restrict__ sorted,
                             int32_t* __restrict__ lb)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    sorted += S.p0;
    lb += S.lb0;
    const int64_t nleaf = level_size(S.L);
    for (int64_t j = (int64_t)z.rank * blockDim.x + threadIdx.x; j <= S.n; j += (int64_t)z.nb * blockDim.x) {
        const int64_t prev = j > 0 ? (int64_t)sorted[j - 1] : -1;
        const int64_t cur = j < S.n ? (int64_t)sorted[j] : nleaf;
        for (int64_t c = prev + 1; c <= cur; c++) lb[c] = (int32_t)j;
    }
}

// largest leaf of each instance into the instance table; schedule: points
__global__ void k_uniform_maxleaf(Sched sc, Inst* __restrict__ I, const int32_t* __restrict__ lb)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    lb += S.lb0;
    int32_t mx = 0;
    for (int64_t c = (int64_t)z.rank * blockDim.x + threadIdx.x; c < level_size(S.L); c += (int64_t)z.nb * blockDim.x)
        mx = max(mx, lb[c + 1] - lb[c]);
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(&I[z.i].maxleaf, mx);
}

__global__ void k_reset_maxleaf(Inst* I, int n_inst)
{
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) I[i].maxleaf = 0;
}

// rectangles of every box; schedule: points (boxes of the instance, grid-stride)
__global__ void k_uniform_rects(Sched sc, const Inst* __restrict__ I, const uint64_t* __restrict__ bbox,
                                double3 root, double* __restrict__ rects)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    rects += 4 * S.b0;
    double x0, y0;
    const double side = root_square(bbox + 4 * z.i, root, x0, y0);
    for (int64_t g = (int64_t)z.rank * blockDim.x + threadIdx.x; g < S.nbox; g += (int64_t)z.nb * blockDim.x) {
        int l = 0;
        while (level_base(l + 1) <= g) l++;
        const int64_t b = g - level_base(l);
        int64_t ix = 0, iy = 0;
        for (int j = 0; j < l; j++) {
            const int64_t d = (b >> (2 * (l - 1 - j))) & 3;
            ix = 2 * ix + (d >> 1);
            iy = 2 * iy + (d & 1);
        }
        const double w = (double)(int64_t(1) << l);
        double* r = rects + 4 * g;
        r[0] = __dadd_rn(x0, __dmul_rn(side, __ddiv_rn((double)ix, w)));
        r[1] = __dadd_rn(x0, __dmul_rn(side, __ddiv_rn((double)(ix + 1), w)));
        r[2] = __dadd_rn(y0, __dmul_rn(side, __ddiv_rn((double)iy, w)));
        r[3] = __dadd_rn(y0, __dmul_rn(side, __ddiv_rn((double)(iy + 1), w)));
    }
}

}  // namespace

// Host tables of one instance (sizes depend on (n, L) only): ones-before tables for depths
// 0 .. 2L-1, node offsets for depths 0 .. 2L, leaf offsets.  Any pointer may be null.
int tree_tables_host(int64_t n, int L, int32_t* ones_before, int32_t* node_off, int32_t* leaf_begin)
{
    std::vector<int64_t> sizes{n}, next;
    int64_t iob = 0, ino = 0;
    for (int d = 0; d <= 2 * L; d++) {
        int64_t o = 0;
        for (int64_t m : sizes) {
            if (node_off) node_off[ino] = (int32_t)o;
            ino++;
            o += m;
        }
        if (node_off) node_off[ino] = (int32_t)o;
        ino++;
        if (d == 2 * L) break;
        int64_t acc = 0;
        for (int64_t m : sizes) {
            if (ones_before) ones_before[iob] = (int32_t)acc;
            iob++;
            acc += m - m / 2;
        }
        next.clear();
        for (int64_t m : sizes) {
            next.push_back(m / 2);
            next.push_back(m - m / 2);
        }
        sizes.swap(next);
    }
    if (leaf_begin) {
        leaf_begin[0] = 0;
        for (size_t i = 0; i < sizes.size(); i++) leaf_begin[i + 1] = leaf_begin[i] + (int32_t)sizes[i];
    }
    return 0;
}

// The instance table of a forest; every size follows from the (n, L) of its instances.
void fill_instances(Inst* out, int n_inst, const int64_t* ns, const int* Ls)
{
    int64_t p0 = 0, b0 = 0, t0 = 0, ob0 = 0, no0 = 0, lb0 = 0;
    for (int i = 0; i < n_inst; i++) {
        Inst& S = out[i];
        S = Inst{};
        S.n = ns[i];
        S.L = Ls[i];
        S.p0 = p0;
        S.b0 = b0;
        S.nbox = level_base(S.L + 1);
        S.o0 = b0 + i;
        S.t0 = t0;
        S.ntiles = (S.n + TILE - 1) / TILE;
        S.ob0 = ob0;
        S.no0 = no0;
        S.lb0 = lb0;
        S.maxleaf = (int32_t)((S.n + level_size(S.L) - 1) / level_size(S.L));
        // the first level whose boxes (at most ceil(n / 4^l) points) fit one block
        S.lg = 0;
        while (S.lg < S.L && (S.n + level_size(S.lg) - 1) / level_size(S.lg) > TREE_LOCAL_CAP) S.lg++;
        p0 += S.n;
        b0 += S.nbox;
        t0 += S.ntiles;
        ob0 += ones_before_offset(2 * S.L);
        no0 += node_offset_base(2 * S.L + 1);
        lb0 += level_size(S.L) + 1;
    }
}

void forest_totals(fmm_tree t)
{
    t->n = t->nbox = t->ntiles = t->n_ob = t->n_no = t->nleaf = 0;
    t->Lmax = 0;
    t->max_tiles = t->max_n = 0;
    for (int i = 0; i < t->n_inst; i++) {
        const Inst& S = t->hinst[i];
        t->n += S.n;
        t->nbox += S.nbox;
        t->ntiles += S.ntiles;
        t->n_ob += ones_before_offset(2 * S.L);
        t->n_no += node_offset_base(2 * S.L + 1);
        t->nleaf += level_size(S.L);
        t->Lmax = std::max(t->Lmax, S.L);
        t->max_tiles = std::max(t->max_tiles, S.ntiles);
        t->max_n = std::max(t->max_n, S.n);
    }
}

int tree_alloc(fmm_tree t, int n_inst, const int64_t* ns, const int* Ls)
{
    t->n_inst = n_inst;
    t->hinst = new (std::nothrow) Inst[n_inst];
    if (!t->hinst) return fail(FMM_ERR_OOM, "host allocation");
    fill_instances(t->hinst, n_inst, ns, Ls);
    forest_totals(t);

    std::vector<int32_t> ob_all(std::max<int64_t>(t->n_ob, 1)), off_all(t->n_no);
    std::vector<int32_t> lb_all(t->nleaf + n_inst);
    for (int i = 0; i < n_inst; i++) {
        const Inst& S = t->hinst[i];
        tree_tables_host(S.n, S.L, ob_all.data() + S.ob0, off_all.data() + S.no0, lb_all.data() + S.lb0);
    }

    auto A = [&](void** p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) return fail(FMM_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        return 0;
    };
    int rc = 0;
    const size_t nb = (size_t)t->nbox, nn = (size_t)t->n, ni = (size_t)n_inst;
    if ((rc = A((void**)&t->dinst, sizeof(Inst) * ni))) return rc;
    if ((rc = A((void**)&t->rects, 32 * nb))) return rc;
    if ((rc = A((void**)&t->centers, 16 * nb))) return rc;
    if ((rc = A((void**)&t->radii, 8 * nb))) return rc;
    if ((rc = A((void**)&t->rad32, 4 * nb))) return rc;
    if ((rc = A((void**)&t->cen_hi, 8 * nb))) return rc;
    if ((rc = A((void**)&t->cen_lo, 8 * nb))) return rc;
    if ((rc = A((void**)&t->perm, 4 * nn))) return rc;
    if ((rc = A((void**)&t->leaf_begin, 4 * lb_all.size()))) return rc;
    if ((rc = A((void**)&t->leaf_of, 4 * nn))) return rc;
    if ((rc = A((void**)&t->cleaf, 4 * nn))) return rc;
    if ((rc = A((void**)&t->xs, 8 * nn))) return rc;
    if ((rc = A((void**)&t->ys, 8 * nn))) return rc;
    if ((rc = A((void**)&t->dxf, 4 * nn))) return rc;
    if ((rc = A((void**)&t->dyf, 4 * nn))) return rc;
    if ((rc = A((void**)&t->keys, 8 * 4 * nn))) return rc;
    if ((rc = A((void**)&t->vals, 4 * 4 * nn))) return rc;
    if ((rc = A((void**)&t->rs_counts, 4 * 2 * BINS * (size_t)t->ntiles))) return rc;
    if ((rc = A((void**)&t->rs_totals, 4 * 2 * BINS * ni))) return rc;
    if ((rc = A((void**)&t->tilecnt, 4 * (size_t)t->ntiles))) return rc;
    if ((rc = A((void**)&t->hflag, 2 * nn))) return rc;
    if ((rc = A((void**)&t->bbox_keys, 32 * ni))) return rc;
    if ((rc = A((void**)&t->ones_before, 4 * ob_all.size()))) return rc;
    if ((rc = A((void**)&t->node_off, 4 * off_all.size()))) return rc;
    if ((rc = A((void**)&t->segs, 4 * 4 * nn))) return rc;
    if ((rc = A((void**)&t->status, 4))) return rc;
    FMM_CUDA(cudaMemcpy(t->dinst, t->hinst, sizeof(Inst) * ni, cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemcpy(t->leaf_begin, lb_all.data(), 4 * lb_all.size(), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemcpy(t->ones_before, ob_all.data(), 4 * ob_all.size(), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemcpy(t->node_off, off_all.data(), 4 * off_all.size(), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemset(t->status, 0, 4));
    if ((rc = tree_kernel_setup())) return rc;
    if ((rc = sched_all(t))) return rc;
    return queues_make(t);
}

// The block-local split's dynamic shared memory is above the default limit of a launch; the
// opt-in holds for the current device from then on.  Called where a tree is created and on the
// first no-allocation build of a device, so never inside a stream capture of a documented use.
int tree_kernel_setup()
{
    FMM_CUDA(cudaFuncSetAttribute(k_split_local, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(LocalSmem)));
    return 0;
}

int tree_build(fmm_tree t, const double* x, const double* y, cudaStream_t s, cudaEvent_t* level_ready)
{
    const int64_t n = t->n;  // total points of the forest
    const int ni = t->n_inst;
    const int L = t->Lmax;
    const unsigned gt = (unsigned)t->s_tiles.blocks, gp = (unsigned)t->s_pts.blocks;
    const Sched st = t->s_tiles.d, sp = t->s_pts.d;
    uint64_t* kx = t->keys;   // x sort: buffers [0, n) and [n, 2n); y sort: [2n, 4n)
    int32_t* vals = t->vals;  // x sort values [0, 2n); y sort values [2n, 4n)
    uint8_t* hx = t->hflag;
    uint8_t* hy = t->hflag + n;
    int32_t *X, *Xo, *Y, *Yo;
    int32_t* Xfinal_seg = nullptr;

    if (t->uniform) {  // the previous build was the uniform grid: balanced leaves again
        for (int i = 0; i < ni; i++) {
            Inst& S = t->hinst[i];
            S.maxleaf = (int32_t)((S.n + level_size(S.L) - 1) / level_size(S.L));
        }
        FMM_CUDA(cudaMemcpy(t->dinst, t->hinst, sizeof(Inst) * ni, cudaMemcpyHostToDevice));
        FMM_CUDA(cudaMemcpyAsync(t->leaf_begin, t->lb_bal, 4 * (size_t)(t->nleaf + ni), cudaMemcpyDeviceToDevice, s));
        t->uniform = false;
    }
    {
        StageScope scope(FMM_STAGE_TREE_SORT, s);
        k_bbox_init<<<1, 256, 0, s>>>(ni, t->bbox_keys); note_launch();
        k_make_keys<<<gp, 256, 0, s>>>(sp, t->dinst, x, y, n, kx, t->bbox_keys, t->status); note_launch();
        k_root_rect<<<1, 256, 0, s>>>(t->dinst, ni, t->bbox_keys, t->rects); note_launch();
        if (level_ready) {  // the geometry of each level as soon as its rectangles exist
            k_geometry_roots<<<1, 256, 0, s>>>(t->dinst, ni, t->rects, t->centers, t->radii, t->rad32, t->cen_hi,
                                               t->cen_lo); note_launch();
            FMM_CUDA(cudaEventRecord(level_ready[0], s));
        }
        FMM_LAUNCH_CHECK("tree: keys");
        // x order and y order of all points, ties by input index (two sorts in one launch sequence)
        int cur = radix_sort<uint64_t>(t, kx, vals, 2 * n, 2, 64, s);
        FMM_LAUNCH_CHECK("tree: radix sort");
        X = vals + (cur ? n : 0);
        Xo = vals + (cur ? 0 : n);
        Y = vals + 2 * n + (cur ? n : 0);
        Yo = vals + 2 * n + (cur ? 0 : n);
    }

    {
        StageScope scope(FMM_STAGE_TREE_SPLIT, s);
        // global passes for levels l < Lg; the geometry of levels <= Lev is complete after them
        // (the rest comes from the block-local split)
        int Lg = 0, Lev = L;
        for (int i = 0; i < ni; i++) {
            const Inst& S = t->hinst[i];
            Lg = std::max(Lg, (int)S.lg);
            if (S.lg < S.L) Lev = std::min(Lev, (int)S.lg);
        }
        // box index carried by every item of X and Y (all in the root at level 0)
        int32_t *XS = t->segs, *XSo = t->segs + n, *YS = t->segs + 2 * n, *YSo = t->segs + 3 * n;
        FMM_CUDA(cudaMemsetAsync(XS, 0, 4 * n, s));
        FMM_CUDA(cudaMemsetAsync(YS, 0, 4 * n, s));
        k_init_hx<<<gp, 256, 0, s>>>(sp, t->dinst, X, hx); note_launch();
        for (int l = 0; l < Lg; l++) {
            // Y: stable partition of each box by its x-half bit; records the y-half bit
            k_part_count<<<gt, TPB, 0, s>>>(st, t->dinst, l, Y, hx, t->tilecnt); note_launch();
            k_part_scatter<<<gt, TPB, 0, s>>>(st, t->dinst, l, 0, Y, YS, Yo, YSo, hx, hy, t->node_off,
                                              t->ones_before, t->tilecnt, t->status); note_launch();
            std::swap(Y, Yo);
            std::swap(YS, YSo);
            // split coordinates and child rectangles of level l
            k_split_rects<<<t->s_split[l].blocks, 128, 0, s>>>(t->s_split[l].d, t->dinst, l, X, Y, x, y,
                                                                t->node_off, t->rects); note_launch();
            if (level_ready) {
                k_geometry_level<<<t->s_split[l].blocks, 128, 0, s>>>(t->s_split[l].d, t->dinst, l + 1, t->rects,
                                                                     t->centers, t->radii, t->rad32, t->cen_hi,
                                                                     t->cen_lo); note_launch();
                if (l + 1 <= Lev) FMM_CUDA(cudaEventRecord(level_ready[l + 1], s));
            }
            // X: stable partition of each x-half by the y-half bit; records the next x-half bit
            k_part_count<<<gt, TPB, 0, s>>>(st, t->dinst, l, X, hy, t->tilecnt); note_launch();
            k_part_scatter<<<gt, TPB, 0, s>>>(st, t->dinst, l, 1, X, XS, Xo, XSo, hy, hx, t->node_off,
                                              t->ones_before, t->tilecnt, t->status); note_launch();
            std::swap(X, Xo);
            std::swap(XS, XSo);
            FMM_LAUNCH_CHECK("tree: level split");
        }
        if (t->s_local.blocks > 0) {  // the levels below lg, one block per box of level lg
            const int smem = (int)sizeof(LocalSmem);  // opted in when the tree was created
            k_split_local<<<(unsigned)t->s_local.blocks, TREE_LOCAL_TPB, smem, s>>>(
                t->s_local.d, t->dinst, X, XS, Y, x, y, t->node_off, t->ones_before, t->leaf_of, t->rects,
                t->centers, t->radii, t->rad32, t->cen_hi, t->cen_lo, level_ready ? 1 : 0, t->status);
            note_launch();
            FMM_LAUNCH_CHECK("tree: block-local split");
        }
        if (level_ready)
            for (int l = Lev + 1; l <= L; l++) FMM_CUDA(cudaEventRecord(level_ready[l], s));
        Xfinal_seg = XS;
    }

    {
        StageScope scope(FMM_STAGE_TREE_FINISH, s);
        // canonical order: the input indices of every leaf in ascending order.  Small leaves are
        // ranked in place (k_leaf_rank); otherwise a stable sort of the input indices by leaf.
        int32_t maxleaf = 0;
        for (int i = 0; i < ni; i++) maxleaf = std::max(maxleaf, t->hinst[i].maxleaf);
        uint32_t* leaf_of = nullptr;
        if (maxleaf <= LEAF_RANK_MAX) {
            k_leaf_rank<<<gp, 256, 0, s>>>(sp, t->dinst, X, Xfinal_seg, t->leaf_begin, t->perm, t->cleaf,
                                           t->status); note_launch();
        } else {
            leaf_of = (uint32_t*)t->leaf_of;
            k_leaf_of<<<gp, 256, 0, s>>>(sp, t->dinst, X, Xfinal_seg, leaf_of); note_launch();
            uint32_t* k32 = (uint32_t*)t->keys;  // reuse the key buffers: [0, n) and [n, 2n)
            int32_t* v32 = t->vals + 2 * n;      // value buffers [2n, 4n)
            const int bits = std::max(8, 2 * L);  // with L = 0 all keys are 0: the order stays the input order
            FMM_CUDA(cudaMemcpyAsync(k32, leaf_of, 4 * n, cudaMemcpyDeviceToDevice, s));
            int c2 = radix_sort<uint32_t>(t, k32, v32, 0, 1, bits, s);
            FMM_CUDA(cudaMemcpyAsync(t->perm, v32 + (c2 ? n : 0), 4 * n, cudaMemcpyDeviceToDevice, s));
        }

        const int64_t nb = t->nbox;
        if (!level_ready)
            k_geometry<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(t->rects, nb, t->centers, t->radii,
                                                                    t->rad32, t->cen_hi, t->cen_lo);
        note_launch();
        k_gather_points<<<gp, 256, 0, s>>>(sp, t->dinst, t->perm, leaf_of, x, y, t->centers,
                                           t->xs, t->ys, t->dxf, t->dyf, t->cleaf); note_launch();
        FMM_LAUNCH_CHECK("tree: canonical order");
    }
    t->built = true;
    return 0;
}

// The uniform-grid mesh in place of the median tree (same handle, same downstream stages), on the
// bounding square or on a given root square (x0, y0, side) shared by all instances: cells
// of every point, a stable sort by cell (ties keep input order), leaf offsets and the largest
// leaf of every instance (read back, so this call synchronises the stream), the rectangles of
// every box, the box geometry and the canonical coordinates.
int tree_build_uniform(fmm_tree t, const double* x, const double* y, const double* root_host, cudaStream_t s)
{
    const double3 root = root_host ? make_double3(root_host[0], root_host[1], root_host[2])
                                   : make_double3(0.0, 0.0, -1.0);
    const int64_t n = t->n;
    const int ni = t->n_inst;
    const int L = t->Lmax;
    const unsigned gp = (unsigned)t->s_pts.blocks;
    const Sched sp = t->s_pts.d;
    if (!t->lb_bal) {  // keep the balanced leaf offsets for a later median build
        if (cudaMalloc((void**)&t->lb_bal, 4 * (size_t)(t->nleaf + ni)) != cudaSuccess)
            return fail(FMM_ERR_OOM, "leaf offsets");
        FMM_CUDA(cudaMemcpyAsync(t->lb_bal, t->leaf_begin, 4 * (size_t)(t->nleaf + ni), cudaMemcpyDeviceToDevice, s));
    }
    uint32_t* leaf_of = (uint32_t*)t->leaf_of;
    {
        StageScope scope(FMM_STAGE_TREE_SORT, s);
        k_bbox_init<<<1, 256, 0, s>>>(ni, t->bbox_keys); note_launch();
        k_make_keys<<<gp, 256, 0, s>>>(sp, t->dinst, x, y, n, t->keys, t->bbox_keys, t->status); note_launch();
        k_uniform_cells<<<gp, 256, 0, s>>>(sp, t->dinst, x, y, t->bbox_keys, root, leaf_of); note_launch();
        FMM_LAUNCH_CHECK("uniform tree: cells");
        uint32_t* k32 = (uint32_t*)t->keys;
        int32_t* v32 = t->vals + 2 * n;
        const int bits = std::max(8, 2 * L);
        FMM_CUDA(cudaMemcpyAsync(k32, leaf_of, 4 * n, cudaMemcpyDeviceToDevice, s));
        const int c2 = radix_sort<uint32_t>(t, k32, v32, 0, 1, bits, s);
        FMM_CUDA(cudaMemcpyAsync(t->perm, v32 + (c2 ? n : 0), 4 * n, cudaMemcpyDeviceToDevice, s));
        k_uniform_lb<<<gp, 256, 0, s>>>(sp, t->dinst, k32 + (c2 ? n : 0), t->leaf_begin); note_launch();
        k_reset_maxleaf<<<1, 256, 0, s>>>(t->dinst, ni); note_launch();
        k_uniform_maxleaf<<<gp, 256, 0, s>>>(sp, t->dinst, t->leaf_begin); note_launch();
        FMM_LAUNCH_CHECK("uniform tree: order");
    }
    {
        StageScope scope(FMM_STAGE_TREE_FINISH, s);
        k_uniform_rects<<<gp, 256, 0, s>>>(sp, t->dinst, t->bbox_keys, root, t->rects); note_launch();
        const int64_t nb = t->nbox;
        k_geometry<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(t->rects, nb, t->centers, t->radii,
                                                                t->rad32, t->cen_hi, t->cen_lo); note_launch();
        k_gather_points<<<gp, 256, 0, s>>>(sp, t->dinst, t->perm, leaf_of, x, y, t->centers,
                                           t->xs, t->ys, t->dxf, t->dyf, t->cleaf); note_launch();
        FMM_LAUNCH_CHECK("uniform tree: geometry");
    }
    // the largest leaves decide the near-field kernels on the host
    FMM_CUDA(cudaStreamSynchronize(s));
    FMM_CUDA(cudaMemcpy(t->hinst, t->dinst, sizeof(Inst) * ni, cudaMemcpyDeviceToHost));
    t->uniform = true;
    t->built = true;
    return 0;
}

}  // namespace fmm
