// Interaction lists on the GPU: the connectivity rule of Section 4 with the theta-criterion
// (Criterion 2.1).
//
// Level by level, every candidate pair (box b, child c of a box of S(parent(b))) is one thread.
// Candidates are enumerated parent by parent, box by box (b = 4 parent + k), then in the order
// of the parent's strong list and the child index, so each box owns a contiguous, ascending run
// of candidates.  One scan of the weak flags then gives every entry its CSR position and every
// box its offsets, whatever the spread of list lengths (balanced trees of clustered points have
// lists from a handful to thousands of entries).  The number of candidates of a level lives in
// device memory, so the kernels use grid-stride loops over a fixed grid and the whole build is
// asynchronous.  Entries beyond the preallocated capacity are dropped and flagged in the status
// word; later levels never read past the capacity.
//
// All instances of a forest are processed by the same launches (a schedule gives every block its
// instance and its rank among that instance's blocks); each instance has its own CSR arrays,
// capacities and scratch, found through the instance tables.
#include <algorithm>
#include <new>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int LT = 256;          // threads per block
constexpr int LI = 8;            // candidates per thread per tile
constexpr int LTILE = LT * LI;   // candidates per tile

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Criterion 2.1 with correctly rounded binary64 operations in a fixed order (no contraction),
// plus disjointness of the two spheres.
__device__ __forceinline__ bool theta_weak(double ax, double ay, double ra, double bx, double by,
                                           double rb, double theta)
{
    double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by);
    double d = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    double R = ra > rb ? ra : rb;
    double r = ra > rb ? rb : ra;
    return (__dadd_rn(R, __dmul_rn(theta, r)) <= __dmul_rn(theta, d)) && (__dadd_rn(R, r) < d);
}

// The same decision taken in binary32 first (float-float centres, binary32 radii).  Every
// binary32 quantity below is within 2^-20 (relative to theta*d + R + theta*r, resp. d + R + r) of
// its binary64 counterpart, so a margin larger than 2^-16 of that scale has the sign the binary64
// test would find; only candidates closer to the boundary take the binary64 test.
__device__ __forceinline__ bool theta_weak_fast(int64_t a, int64_t b, const float* __restrict__ chi,
                                                const float* __restrict__ clo,
                                                const float* __restrict__ rad32, const double* __restrict__ cen,
                                                const double* __restrict__ rad, float th32, double theta)
{
    const float2 ha = *(const float2*)(chi + 2 * a), hb = *(const float2*)(chi + 2 * b);
    const float2 la = *(const float2*)(clo + 2 * a), lb = *(const float2*)(clo + 2 * b);
    const float dx = (ha.x - hb.x) + (la.x - lb.x), dy = (ha.y - hb.y) + (la.y - lb.y);
    const float d = sqrtf(dx * dx + dy * dy);
    const float ra = rad32[a], rb = rad32[b];
    const float R = fmaxf(ra, rb), r = fminf(ra, rb);
    const float m1 = th32 * d - (R + th32 * r), s1 = th32 * d + R + th32 * r;
    const float m2 = d - (R + r), s2 = d + R + r;
    const float eps = 1.0f / 65536.0f;
    if (fabsf(m1) > eps * s1 && fabsf(m2) > eps * s2) return m1 >= 0.f && m2 > 0.f;
    return theta_weak(cen[2 * a], cen[2 * a + 1], rad[a], cen[2 * b], cen[2 * b + 1], rad[b], theta);
}

// Criterion 2.1 with the roles of the radii exchanged (Section 4's finest-level optimisation):
// r + theta*R <= theta*d, disjoint spheres; binary64 in the same fixed order as theta_weak.
__device__ __forceinline__ bool theta_swapped(double ax, double ay, double ra, double bx, double by,
                                              double rb, double theta)
{
    double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by);
    double d = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    double R = ra > rb ? ra : rb;
    double r = ra > rb ? rb : ra;
    return (__dadd_rn(r, __dmul_rn(theta, R)) <= __dmul_rn(theta, d)) && (__dadd_rn(R, r) < d);
}

// The same two-stage evaluation as theta_weak_fast.
__device__ __forceinline__ bool theta_swapped_fast(int64_t a, int64_t b, const float* __restrict__ chi,
                                                   const float* __restrict__ clo,
                                                   const float* __restrict__ rad32, const double* __restrict__ cen,
                                                   const double* __restrict__ rad, float th32, double theta)
{
    const float2 ha = *(const float2*)(chi + 2 * a), hb = *(const float2*)(chi + 2 * b);
    const float2 la = *(const float2*)(clo + 2 * a), lb = *(const float2*)(clo + 2 * b);
    const float dx = (ha.x - hb.x) + (la.x - lb.x), dy = (ha.y - hb.y) + (la.y - lb.y);
    const float d = sqrtf(dx * dx + dy * dy);
    const float ra = rad32[a], rb = rad32[b];
    const float R = fmaxf(ra, rb), r = fminf(ra, rb);
    const float m1 = th32 * d - (r + th32 * R), s1 = th32 * d + r + th32 * R;
    const float m2 = d - (R + r), s2 = d + R + r;
    const float eps = 1.0f / 65536.0f;
    if (fabsf(m1) > eps * s1 && fabsf(m2) > eps * s2) return m1 >= 0.f && m2 > 0.f;
    return theta_swapped(cen[2 * a], cen[2 * a + 1], rad[a], cen[2 * b], cen[2 * b + 1], rad[b], theta);
}

// Optional list variants (Section 4's structural optimisations).
struct ListOpt {
    uint32_t* tiledrop;  // per candidate tile: siblings covered by a parent entry
    uint32_t* tileswap;  // per candidate tile: finest-level pairs moved to the exchange lists
    int32_t* xoff;       // role-exchange lists: offsets over all boxes (layout of woff)
    int32_t* xidx;       // entries (layout and capacity of the strong lists)
    int32_t* xtgt;       // their targets (global leaf ids)
};

// One instance's view of the list arrays (pointers already offset to the instance).
struct LView {
    int32_t *woff, *soff, *widx, *wrow, *sidx, *stgt;
    uint8_t* flags;
    uint32_t* tilecnt;
    int64_t wcap, scap;
};

__device__ __forceinline__ LView lview(const Inst& S, const LInst& T, int32_t* woff, int32_t* soff,
                                       int32_t* widx, int32_t* wrow, int32_t* sidx, int32_t* stgt,
                                       uint8_t* flags, uint32_t* tilecnt)
{
    LView v;
    v.woff = woff + S.o0;
    v.soff = soff + S.o0;
    v.widx = widx + T.w0;
    v.wrow = wrow + (T.w0 >> 3);
    v.sidx = sidx + T.s0;
    v.stgt = stgt + T.s0;
    v.flags = flags + T.f0;
    v.tilecnt = tilecnt + T.c0;
    v.wcap = T.wcap;
    v.scap = T.scap;
    return v;
}

#define LIST_ARGS                                                                                 \
    const Inst *__restrict__ I, const LInst *__restrict__ LIs, int32_t *woff, int32_t *soff,     \
        int32_t *widx, int32_t *wrow, int32_t *sidx, int32_t *stgt, uint8_t *flags,               \
        uint32_t *tilecnt
#define LIST_VIEW(i) lview(I[i], LIs[i], woff, soff, widx, wrow, sidx, stgt, flags, tilecnt)

__global__ void k_lists_root(LIST_ARGS, int n_inst)
{
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
        const LView v = lview(I[i], LIs[i], woff, soff, widx, wrow, sidx, stgt, flags, tilecnt);
        v.woff[0] = 0;
        v.woff[1] = 0;
        v.soff[0] = 0;
        v.soff[1] = 1;
        v.sidx[0] = 0;
        v.stgt[0] = 0;
    }
}

// Parent-level strong entries of level l-1 that lie within the capacity: [S0, S1).
struct LevelCands {
    int64_t S0, S1;
    __device__ __forceinline__ int64_t count() const { return 16 * (S1 - S0); }
};

__device__ __forceinline__ LevelCands level_cands(const int32_t* soff, int l, int64_t scap)
{
    const int64_t pb0 = level_base(l - 1), np = level_size(l - 1);
    LevelCands c;
    c.S0 = min((int64_t)soff[pb0], scap);
    c.S1 = min((int64_t)soff[pb0 + np], scap);
    if (c.S1 < c.S0) c.S1 = c.S0;
    return c;
}

// Parent offsets of one tile.  Every parent owns 16 * |S(parent)| >= 16 consecutive candidates,
// so a tile of LTILE candidates touches at most LTILE / 16 + 2 parents: their clamped strong-list
// offsets are staged in shared memory once per tile and every candidate is decoded there.
constexpr int TP_MAX = LTILE / 16 + 2;

struct TileParents {
    int64_t p0;               // first parent of the tile
    int np;                   // parents staged
    int64_t off[TP_MAX + 1];  // clamped soff of parents p0 .. p0 + np
};

__device__ __forceinline__ int64_t find_parent(const int32_t* __restrict__ soff, int64_t pb0, int64_t np,
                                               int64_t scap, int64_t S0, int64_t t)
{
    int64_t lo = 0, hi = np - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (16 * (min((int64_t)soff[pb0 + mid], scap) - S0) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Called by the whole block: stage the parents of candidates [t0, t1).
__device__ __forceinline__ void stage_parents(TileParents& tp, const int32_t* __restrict__ soff, int l,
                                              int64_t scap, const LevelCands& lc, int64_t t0, int64_t t1)
{
    const int64_t pb0 = level_base(l - 1), np = level_size(l - 1);
    __shared__ int64_t ends[2];
    if (threadIdx.x < 2) ends[threadIdx.x] = find_parent(soff, pb0, np, scap, lc.S0, threadIdx.x ? t1 - 1 : t0);
    __syncthreads();
    const int64_t p0 = ends[0], p1 = ends[1];
    const int cnt = (int)(p1 - p0 + 1);
    for (int i = threadIdx.x; i <= cnt; i += blockDim.x) tp.off[i] = min((int64_t)soff[pb0 + p0 + i], scap);
    if (threadIdx.x == 0) {
        tp.p0 = p0;
        tp.np = cnt;
    }
    __syncthreads();
}

// Decode candidate t of level l: box b (within-level), candidate c (within-level), and whether t
// is the first candidate of its box.
__device__ __forceinline__ void decode(const TileParents& tp, const int32_t* __restrict__ sidx,
                                       const LevelCands& lc, int64_t t, int64_t& b, int64_t& c, bool& first)
{
    int lo = 0, hi = tp.np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (16 * (tp.off[mid] - lc.S0) <= t) lo = mid;
        else hi = mid - 1;
    }
    const int64_t s0 = tp.off[lo];
    const uint32_t m = (uint32_t)(tp.off[lo + 1] - s0);  // >= 1 for the parent that owns t
    const uint32_t tq = (uint32_t)(t - 16 * (s0 - lc.S0));
    const uint32_t k = tq / (4 * m), r = tq - k * 4 * m;
    b = 4 * (tp.p0 + lo) + k;
    c = 4 * (int64_t)sidx[s0 + (r >> 2)] + (r & 3);
    first = (r == 0);
}

// Candidate flags: 0 strong, 1 weak.  With parent-level interactions (PAR, Section 4's optional
// step) four weak siblings c = 4k .. 4k+3 of one target box whose parent k also satisfies the
// criterion with the target become one entry: 2 on the first (the entry names the parent), 3 on
// the other three (no entry).  The four children of a source box are candidates 4q .. 4q+3,
// which sit in lanes 4q' .. 4q'+3 of one warp (tiles, rows and boxes all start at multiples of
// 4), so one ballot tells each lane about its quad.  With the role exchange (SWP) a strong
// candidate of an instance's finest level that passes the exchanged criterion is flagged 4 (the
// target is the smaller leaf: P2L) or 5 (the larger: M2P) and goes to the exchange lists.
// schedule: candidate tiles of level l
template <bool PAR, bool SWP>
__global__ void __launch_bounds__(LT) k_lists_flags(Sched sc, LIST_ARGS, ListOpt opt, int l,
                                                    const double* __restrict__ cen,
                                                    const double* __restrict__ rad,
                                                    const float* __restrict__ chi,
                                                    const float* __restrict__ clo,
                                                    const float* __restrict__ rad32, double theta)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    if (l > S.L) return;
    const LView v = LIST_VIEW(z.i);
    const bool fin = SWP && l == S.L;
    cen += 2 * S.b0;
    rad += S.b0;
    chi += 2 * S.b0;
    clo += 2 * S.b0;
    rad32 += S.b0;
    __shared__ uint32_t wsum[LT / 32], dsum[LT / 32], xsum[LT / 32];
    __shared__ TileParents tp;
    const LevelCands lc = level_cands(v.soff, l, v.scap);
    const int64_t nc = lc.count();
    const int64_t ntiles = (nc + LTILE - 1) / LTILE;
    const int64_t base = level_base(l), pbase = level_base(l - 1);
    const int lane = threadIdx.x & 31;
    for (int64_t tile = z.rank; tile < ntiles; tile += z.nb) {
        stage_parents(tp, v.soff, l, v.scap, lc, tile * LTILE, min(nc, (tile + 1) * LTILE));
        uint32_t cnt = 0, drop = 0, swp = 0;
#pragma unroll 4
        for (int j = 0; j < LI; j++) {
            const int64_t t = tile * LTILE + (int64_t)j * LT + threadIdx.x;
            int64_t b = 0, c = 0;
            bool w = false;
            if (t < nc) {
                bool first;
                decode(tp, v.sidx, lc, t, b, c, first);
                w = theta_weak_fast(base + b, base + c, chi, clo, rad32, cen, rad, (float)theta, theta);
            }
            uint8_t f = w ? 1 : 0;
            if (PAR) {
                const unsigned q = __ballot_sync(0xffffffffu, w) >> (lane & ~3) & 0xFu;
                bool m = false;
                if (q == 0xFu && (lane & 3) == 0)
                    m = theta_weak_fast(base + b, pbase + (c >> 2), chi, clo, rad32, cen, rad, (float)theta, theta);
                if (__ballot_sync(0xffffffffu, m) >> (lane & ~3) & 1u) f = (lane & 3) ? 3 : 2;
                drop += f == 3;
            }
            if (SWP && fin && t < nc && f == 0 &&
                theta_swapped_fast(base + b, base + c, chi, clo, rad32, cen, rad, (float)theta, theta)) {
                f = rad[base + b] > rad[base + c] ? 5 : 4;
                swp++;
            }
            if (t < nc) v.flags[t] = f;
            cnt += f == 1 || f == 2;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            if (PAR) drop += __shfl_xor_sync(0xffffffffu, drop, o);
            if (SWP) swp += __shfl_xor_sync(0xffffffffu, swp, o);
        }
        if (lane == 0) {
            wsum[threadIdx.x >> 5] = cnt;
            dsum[threadIdx.x >> 5] = drop;
            xsum[threadIdx.x >> 5] = swp;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t s = 0, d = 0, x = 0;
            for (int w = 0; w < LT / 32; w++) {
                s += wsum[w];
                d += dsum[w];
                x += xsum[w];
            }
            v.tilecnt[tile] = s;
            if (PAR) opt.tiledrop[LIs[z.i].c0 + tile] = d;
            if (SWP) opt.tileswap[LIs[z.i].c0 + tile] = x;
        }
        __syncthreads();
    }
}

// In-place exclusive scan of a[0 .. n) by the whole block; returns the total.
__device__ int64_t block_exclusive_scan(uint32_t* a, int64_t n)
{
    __shared__ int64_t wt[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < n; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        int64_t val = i < n ? a[i] : 0, x = val;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wt[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t s = lane < nw ? wt[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            if (lane < nw) wt[lane] = s;
        }
        __syncthreads();
        const int64_t before = w ? wt[w - 1] : 0, tot = wt[nw - 1];
        if (i < n) a[i] = (uint32_t)(carry + before + x - val);
        carry += tot;
        __syncthreads();
    }
    return carry;
}

// Exclusive scan of the weak counts per tile (and of the dropped siblings with PAR, of the
// exchanged pairs at the finest level with SWP); writes the level totals into the offsets.
// One block per instance.
template <bool PAR, bool SWP>
__global__ void __launch_bounds__(1024) k_lists_scan(LIST_ARGS, ListOpt opt, int l)
{
    const Inst S = I[blockIdx.x];
    if (l > S.L) return;
    const LView v = LIST_VIEW(blockIdx.x);
    const bool fin = SWP && l == S.L;
    const LevelCands lc = level_cands(v.soff, l, v.scap);
    const int64_t nc = lc.count();
    const int64_t ntiles = (nc + LTILE - 1) / LTILE;
    const int64_t c0 = LIs[blockIdx.x].c0;
    const int64_t nweak = block_exclusive_scan(v.tilecnt, ntiles);
    const int64_t ndrop = PAR ? block_exclusive_scan(opt.tiledrop + c0, ntiles) : 0;
    const int64_t nswap = fin ? block_exclusive_scan(opt.tileswap + c0, ntiles) : 0;
    if (threadIdx.x == 0) {
        const int64_t base = level_base(l), nb = level_size(l);
        const int64_t W0 = v.woff[base], S0 = v.soff[base];
        v.woff[base + nb] = (int32_t)min(W0 + nweak, (int64_t)INT32_MAX);
        v.soff[base + nb] = (int32_t)min(S0 + (nc - nweak - ndrop - nswap), (int64_t)INT32_MAX);
        if (fin) opt.xoff[S.o0 + base + nb] = (int32_t)min(nswap, (int64_t)INT32_MAX);
    }
}

// Scatter the candidates into the weak, strong (and exchange) lists and write the box offsets.
// The tile prefix of weak flags is tilecnt[tile] (of dropped siblings tiledrop[tile], of
// exchanged pairs tileswap[tile]); the strong prefix is the rest.
// schedule: candidate tiles of level l
template <bool PAR, bool SWP>
__global__ void __launch_bounds__(LT) k_lists_fill(Sched sc, LIST_ARGS, ListOpt opt, int l)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    if (l > S.L) return;
    const LView v = LIST_VIEW(z.i);
    const bool fin = SWP && l == S.L;
    constexpr int NC = 1 + PAR + SWP;  // prefix counters: weak, dropped, exchanged
    __shared__ uint32_t csum[NC][LI][LT / 32];
    __shared__ TileParents tp;
    const LevelCands lc = level_cands(v.soff, l, v.scap);
    const int64_t nc = lc.count();
    const int64_t ntiles = (nc + LTILE - 1) / LTILE;
    const int64_t base = level_base(l);
    const int64_t W0 = v.woff[base], S0 = v.soff[base];
    const int64_t c0 = LIs[z.i].c0;
    int32_t* xoff = SWP ? opt.xoff + S.o0 : nullptr;
    int32_t* xidx = SWP ? opt.xidx + LIs[z.i].s0 : nullptr;
    int32_t* xtgt = SWP ? opt.xtgt + LIs[z.i].s0 : nullptr;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    for (int64_t tile = z.rank; tile < ntiles; tile += z.nb) {
        stage_parents(tp, v.soff, l, v.scap, lc, tile * LTILE, min(nc, (tile + 1) * LTILE));
        uint8_t f[LI];
        uint32_t pre[NC][LI];
#pragma unroll
        for (int j = 0; j < LI; j++) {
            const int64_t t = tile * LTILE + (int64_t)j * LT + threadIdx.x;
            f[j] = t < nc ? v.flags[t] : 0;
#pragma unroll
            for (int k = 0; k < NC; k++) {
                // counter k: 0 weak (1, 2), then dropped (3) if PAR, then exchanged (4, 5) if SWP
                const int kind = k == 0 ? 0 : (PAR && k == 1) ? 1 : 2;
                const bool in = kind == 0 ? (f[j] == 1 || f[j] == 2) : kind == 1 ? f[j] == 3 : f[j] >= 4;
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                pre[k][j] = __popc(bal & lt);
                if (lane == 0) csum[k][j][w] = __popc(bal);
            }
        }
        __syncthreads();
        // exclusive prefix in (row j, warp) order = candidate order inside the tile: warp 0 scans
        // the LI x (LT / 32) = 64 counts of each counter (two per lane) in place
        static_assert(LI * (LT / 32) == 64, "the prefix scan takes two counts per lane");
        if (w == 0) {
#pragma unroll
            for (int k = 0; k < NC; k++) {
                uint32_t* a = &csum[k][0][0];
                const uint32_t c0v = a[2 * lane], c1v = a[2 * lane + 1];
                uint32_t x = c0v + c1v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                const uint32_t ex = x - (c0v + c1v);
                a[2 * lane] = ex;
                a[2 * lane + 1] = ex + c0v;
            }
        }
        __syncthreads();
        uint32_t run[NC];
        run[0] = v.tilecnt[tile];
        if (PAR) run[1] = opt.tiledrop[c0 + tile];
        if (SWP) run[NC - 1] = fin ? opt.tileswap[c0 + tile] : 0;
#pragma unroll
        for (int j = 0; j < LI; j++) {
            uint32_t before[NC];
#pragma unroll
            for (int k = 0; k < NC; k++) before[k] = run[k] + csum[k][j][w];
            const int64_t t = tile * LTILE + (int64_t)j * LT + threadIdx.x;
            if (t < nc) {
                int64_t b, c;
                bool first;
                decode(tp, v.sidx, lc, t, b, c, first);
                const int64_t wpre = (int64_t)before[0] + pre[0][j];  // weak entries before t
                const int64_t dpre = PAR ? (int64_t)before[1] + pre[1][j] : 0;
                const int64_t xpre = SWP ? (int64_t)before[NC - 1] + pre[NC - 1][j] : 0;
                const int64_t spre = t - wpre - dpre - xpre;  // strong entries before t
                if (first) {
                    v.woff[base + b] = (int32_t)min(W0 + wpre, (int64_t)INT32_MAX);
                    v.soff[base + b] = (int32_t)min(S0 + spre, (int64_t)INT32_MAX);
                    if (fin) xoff[base + b] = (int32_t)min(xpre, (int64_t)INT32_MAX);
                }
                if (PAR && f[j] == 3) {
                    // a sibling covered by its parent's entry
                } else if (SWP && f[j] >= 4) {
                    if (xpre < v.scap) {
                        xidx[xpre] = f[j] == 5 ? (int32_t)c | SWAP_M2P : (int32_t)c;
                        xtgt[xpre] = (int32_t)(base + b);
                    }
                } else if (f[j]) {
                    const int64_t pos = W0 + wpre;
                    if (pos < v.wcap) {
                        v.widx[pos] = f[j] == 2 ? (int32_t)(c >> 2) | PARENT_FLAG : (int32_t)c;
                        if ((pos & 7) == 0) v.wrow[pos >> 3] = (int32_t)(base + b);
                    }
                } else {
                    const int64_t pos = S0 + spre;
                    if (pos < v.scap) {
                        v.sidx[pos] = (int32_t)c;
                        v.stgt[pos] = (int32_t)(base + b);
                    }
                }
            }
        }
        __syncthreads();
    }
}

__global__ void k_lists_check(LIST_ARGS, int n_inst, const int32_t* xoff, int32_t* status)
{
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
        const Inst& S = I[i];
        const LView v = lview(S, LIs[i], woff, soff, widx, wrow, sidx, stgt, flags, tilecnt);
        const int32_t W = v.woff[S.nbox], Sx = v.soff[S.nbox];
        const int32_t X = xoff ? xoff[S.o0 + S.nbox] : 0;
        if ((int64_t)W > v.wcap || (int64_t)Sx > v.scap || W == INT32_MAX || Sx == INT32_MAX ||
            (int64_t)X > v.scap || X == INT32_MAX)
            atomicOr(status, ST_CAPACITY);
    }
}

}  // namespace

int64_t lists_flag_bytes(int64_t scap) { return 16 * scap + LTILE; }
int64_t lists_tile_words(int64_t scap) { return (16 * scap + LTILE - 1) / LTILE + 1; }


// Capacities are split over the instances in proportion to their box counts (at least 16 weak and
// 8 strong entries per box).
int lists_alloc(fmm_tree t, fmm_lists l, const int64_t* weak_capacity, const int64_t* strong_capacity)
{
    const int ni = t->n_inst;
    l->hlinst = new (std::nothrow) LInst[ni];
    if (!l->hlinst) return fail(FMM_ERR_OOM, "host allocation");
    int64_t w0 = 0, s0 = 0, f0 = 0, c0 = 0;
    for (int i = 0; i < ni; i++) {
        LInst& T = l->hlinst[i];
        T.wcap = (weak_capacity[i] + 7) & ~int64_t(7);  // rows of eight entries (wrow)
        T.scap = strong_capacity[i];
        T.w0 = w0;
        T.s0 = s0;
        T.f0 = f0;
        T.c0 = c0;
        w0 += T.wcap;
        s0 += T.scap;
        f0 += lists_flag_bytes(T.scap);
        c0 += lists_tile_words(T.scap);
    }
    if (w0 >= INT32_MAX || s0 >= INT32_MAX) return fail(FMM_ERR_ARG, "capacity must be below 2^31 - 1");
    l->wcap = w0;
    l->scap = s0;
    const int64_t noff = t->nbox + ni;
    bool ok = cudaMalloc((void**)&l->dlinst, sizeof(LInst) * ni) == cudaSuccess &&
              cudaMalloc((void**)&l->woff, 4 * noff) == cudaSuccess &&
              cudaMalloc((void**)&l->soff, 4 * noff) == cudaSuccess &&
              cudaMalloc((void**)&l->widx, 4 * std::max<int64_t>(w0, 1)) == cudaSuccess &&
              cudaMalloc((void**)&l->wrow, 4 * (w0 / 8 + 1)) == cudaSuccess &&
              cudaMalloc((void**)&l->rowtgt, 4 * std::max<int64_t>(w0, 1)) == cudaSuccess &&
              cudaMalloc((void**)&l->sidx, 4 * std::max<int64_t>(s0, 1)) == cudaSuccess &&
              cudaMalloc((void**)&l->stgt, 4 * std::max<int64_t>(s0, 1)) == cudaSuccess &&
              cudaMalloc((void**)&l->flags, f0) == cudaSuccess &&
              cudaMalloc((void**)&l->tilecnt, 4 * c0) == cudaSuccess &&
              cudaMalloc((void**)&l->status, 4) == cudaSuccess;
    if (!ok) return fail(FMM_ERR_OOM, "list storage");
    FMM_CUDA(cudaMemcpy(l->dlinst, l->hlinst, sizeof(LInst) * ni, cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemset(l->status, 0, 4));
    return 0;
}

int lists_build(fmm_tree t, fmm_lists li, double theta, cudaStream_t s, const cudaEvent_t* level_ready)
{
    const int L = t->Lmax, ni = t->n_inst;
    StageScope scope(FMM_STAGE_LISTS, s);
    const bool par = (li->mode & FMM_LISTS_PARENTS) != 0, swp = (li->mode & FMM_LISTS_EXCHANGE) != 0;
    const ListOpt opt{li->tiledrop, li->tileswap, li->xoff, li->xidx, li->xtgt};
#define LARGS t->dinst, li->dlinst, li->woff, li->soff, li->widx, li->wrow, li->sidx, li->stgt, li->flags, li->tilecnt
    // with level_ready this stream runs beside the tree build: event 0 also orders these writes
    // after the earlier work of the tree's stream (which may still read the previous lists)
    if (level_ready) FMM_CUDA(cudaStreamWaitEvent(s, level_ready[0], 0));
    k_lists_root<<<1, 256, 0, s>>>(LARGS, ni); note_launch();
    // exchange offsets below the finest level stay 0
    if (swp) FMM_CUDA(cudaMemsetAsync(li->xoff, 0, 4 * (size_t)(t->nbox + ni), s));
    for (int l = 1; l <= L; l++) {
        // a single instance keeps the fixed grid of the grid-stride loops (its candidate count
        // is only known on the device); a forest shares blocks in proportion to 4^l
        const SchedH& sh = t->s_lists[l];
        const unsigned g = ni == 1 ? 152 * 8 : (unsigned)sh.blocks;
        if (level_ready) FMM_CUDA(cudaStreamWaitEvent(s, level_ready[l], 0));
#define LEVEL(PAR, SWP)                                                                                   \
    do {                                                                                                  \
        k_lists_flags<PAR, SWP><<<g, LT, 0, s>>>(sh.d, LARGS, opt, l, t->centers, t->radii, t->cen_hi,   \
                                                 t->cen_lo, t->rad32, theta); note_launch();             \
        k_lists_scan<PAR, SWP><<<ni, 1024, 0, s>>>(LARGS, opt, l); note_launch();                        \
        k_lists_fill<PAR, SWP><<<g, LT, 0, s>>>(sh.d, LARGS, opt, l); note_launch();                     \
    } while (0)
        if (par && swp) LEVEL(true, true);
        else if (par) LEVEL(true, false);
        else if (swp) LEVEL(false, true);
        else LEVEL(false, false);
#undef LEVEL
        FMM_LAUNCH_CHECK("lists");
    }
    k_lists_check<<<1, 256, 0, s>>>(LARGS, ni, swp ? li->xoff : nullptr, li->status); note_launch();
#undef LARGS
    FMM_LAUNCH_CHECK("lists: check");
    li->theta = theta;
    li->built = true;
    return 0;
}

}  // namespace fmm
