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
constexpr int QI = LI / 4;       // quads (four consecutive candidates) per thread per tile

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

// A box's binary32 view: float-float centre and binary32 radius.
struct BoxG {
    float2 h, l;
    float r;
};

__device__ __forceinline__ BoxG box_geom(int64_t g, const float* __restrict__ chi, const float* __restrict__ clo,
                                         const float* __restrict__ rad32)
{
    BoxG B;
    B.h = *(const float2*)(chi + 2 * g);
    B.l = *(const float2*)(clo + 2 * g);
    B.r = rad32[g];
    return B;
}

// Criterion 2.1 (SW = false) or its exchanged form (SW = true) decided in binary32 first, from
// float-float centres and binary32 radii already loaded.  Every binary32 quantity below is within
// 2^-20 (relative to theta*d + R + theta*r, resp. d + R + r) of its binary64 counterpart, so a
// margin larger than 2^-16 of that scale has the sign the binary64 test would find; only
// candidates closer to the boundary take the binary64 test (theta_weak / theta_swapped, by index).
template <bool SW>
__device__ __forceinline__ bool crit_fast(const BoxG& A, const BoxG& B, int64_t a, int64_t b,
                                          const double* __restrict__ cen, const double* __restrict__ rad,
                                          float th32, double theta)
{
    const float dx = (A.h.x - B.h.x) + (A.l.x - B.l.x), dy = (A.h.y - B.h.y) + (A.l.y - B.l.y);
    const float d = sqrtf(dx * dx + dy * dy);
    const float R = fmaxf(A.r, B.r), r = fminf(A.r, B.r);
    const float m1 = SW ? th32 * d - (r + th32 * R) : th32 * d - (R + th32 * r);
    const float s1 = SW ? th32 * d + r + th32 * R : th32 * d + R + th32 * r;
    const float m2 = d - (R + r), s2 = d + R + r;
    const float eps = 1.0f / 65536.0f;
    if (fabsf(m1) > eps * s1 && fabsf(m2) > eps * s2) return m1 >= 0.f && m2 > 0.f;
    return SW ? theta_swapped(cen[2 * a], cen[2 * a + 1], rad[a], cen[2 * b], cen[2 * b + 1], rad[b], theta)
              : theta_weak(cen[2 * a], cen[2 * a + 1], rad[a], cen[2 * b], cen[2 * b + 1], rad[b], theta);
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

// The parent owning candidate t: the largest p < np with 16 * (soff[pb0 + p] - S0) <= t (soff
// clamped to the capacity), found by a whole warp.  Each round the 32 lanes probe 32 evenly
// spaced parents of the remaining range at once and one ballot narrows it about 32-fold, so a
// level of 4^l parents takes about l / 2.5 rounds of loads instead of 2l dependent ones.  Every
// lane returns the result.
__device__ __forceinline__ int64_t find_parent_warp(const int32_t* __restrict__ soff, int64_t pb0, int64_t np,
                                                    int64_t scap, int64_t S0, int64_t t)
{
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = np - 1;  // the answer lies in [lo, hi]; parent 0 always qualifies
    while (hi > lo) {
        const int64_t span = hi - lo;
        // probes lo < m_0 <= m_1 <= ... <= m_31 = hi; the qualifying ones form a prefix of lanes
        const int64_t m = lo + (span * (lane + 1) + 31) / 32;
        const bool ok = 16 * (min((int64_t)soff[pb0 + m], scap) - S0) <= t;
        const int c = __popc(__ballot_sync(0xffffffffu, ok));
        const int64_t nlo = c ? lo + (span * c + 31) / 32 : lo;              // last qualifying probe
        const int64_t nhi = c < 32 ? lo + (span * (c + 1) + 31) / 32 - 1 : hi;  // below the first failing one
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// Called by the whole block: stage the parents of candidates [t0, t1).
__device__ __forceinline__ void stage_parents(TileParents& tp, const int32_t* __restrict__ soff, int l,
                                              int64_t scap, const LevelCands& lc, int64_t t0, int64_t t1)
{
    const int64_t pb0 = level_base(l - 1), np = level_size(l - 1);
    __shared__ int64_t ends[2];
    if (threadIdx.x < 64) {  // warps 0 and 1: the parents of the tile's first and last candidates
        const int64_t e = find_parent_warp(soff, pb0, np, scap, lc.S0, threadIdx.x < 32 ? t0 : t1 - 1);
        if ((threadIdx.x & 31) == 0) ends[threadIdx.x >> 5] = e;
    }
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
// the other three (no entry).  The four children of a source box are candidates 4q .. 4q+3
// (tiles and boxes start at multiples of 4), and one thread decides such a quad, so the parent
// test needs no communication between threads.  With the role exchange (SWP) a strong
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
    const float th32 = (float)theta;
    for (int64_t tile = z.rank; tile < ntiles; tile += z.nb) {
        stage_parents(tp, v.soff, l, v.scap, lc, tile * LTILE, min(nc, (tile + 1) * LTILE));
        uint32_t cnt = 0, drop = 0, swp = 0;
        // each thread takes whole quads: the four children c .. c + 3 of one source box against
        // one target box b (candidates 4q .. 4q + 3), so the decode, the target's geometry and
        // the parent-level test are done once per quad
#pragma unroll
        for (int j = 0; j < QI; j++) {
            const int64_t t = 4 * (tile * (LTILE / 4) + (int64_t)j * LT + threadIdx.x);
            if (t >= nc) continue;
            int64_t b, c;
            bool first;
            decode(tp, v.sidx, lc, t, b, c, first);
            const int64_t gb = base + b, gc = base + c;
            const BoxG T = box_geom(gb, chi, clo, rad32);
            BoxG C[4];
            uint32_t f[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                C[i] = box_geom(gc + i, chi, clo, rad32);
                f[i] = crit_fast<false>(T, C[i], gb, gc + i, cen, rad, th32, theta) ? 1u : 0u;
            }
            if (PAR && (f[0] & f[1] & f[2] & f[3]) &&
                crit_fast<false>(T, box_geom(pbase + (c >> 2), chi, clo, rad32), gb, pbase + (c >> 2), cen, rad,
                                 th32, theta)) {
                f[0] = 2;
                f[1] = f[2] = f[3] = 3;
                drop += 3;
            }
            if (SWP && fin) {
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if (f[i] == 0 && crit_fast<true>(T, C[i], gb, gc + i, cen, rad, th32, theta)) {
                        f[i] = rad[gb] > rad[gc + i] ? 5 : 4;
                        swp++;
                    }
            }
            *(uint32_t*)(v.flags + t) = f[0] | f[1] << 8 | f[2] << 16 | f[3] << 24;
#pragma unroll
            for (int i = 0; i < 4; i++) cnt += f[i] == 1 || f[i] == 2;
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

// Whether flag f counts for counter kind 0 (weak entry: 1, 2), 1 (sibling covered by its
// parent's entry: 3) or 2 (exchanged pair: 4, 5).
__device__ __forceinline__ uint32_t flag_in(uint32_t f, int kind)
{
    return kind == 0 ? (f == 1 || f == 2) : kind == 1 ? f == 3 : f >= 4;
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
    __shared__ uint32_t csum[NC][QI][LT / 32];
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
    for (int64_t tile = z.rank; tile < ntiles; tile += z.nb) {
        stage_parents(tp, v.soff, l, v.scap, lc, tile * LTILE, min(nc, (tile + 1) * LTILE));
        // per quad (four consecutive candidates, as the flag pass made them): its flags, its count
        // of each counter and the exclusive prefix of those counts over the warp's lanes
        uint32_t fw[QI];
        uint32_t pre[NC][QI];
#pragma unroll
        for (int j = 0; j < QI; j++) {
            const int64_t t = 4 * (tile * (LTILE / 4) + (int64_t)j * LT + threadIdx.x);
            fw[j] = t < nc ? *(const uint32_t*)(v.flags + t) : 0u;
#pragma unroll
            for (int k = 0; k < NC; k++) {
                // counter k: 0 weak (1, 2), then dropped (3) if PAR, then exchanged (4, 5) if SWP
                const int kind = k == 0 ? 0 : (PAR && k == 1) ? 1 : 2;
                uint32_t cq = 0;
#pragma unroll
                for (int i = 0; i < 4; i++) cq += flag_in(fw[j] >> (8 * i) & 0xffu, kind);
                uint32_t x = cq;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                pre[k][j] = x - cq;
                if (lane == 31) csum[k][j][w] = x;
            }
        }
        __syncthreads();
        // exclusive prefix of the warp totals in (row j, warp) order = candidate order inside the
        // tile: warp 0 scans the QI x (LT / 32) = 16 totals of each counter in place
        static_assert(QI * (LT / 32) <= 32, "one warp total per lane");
        if (w == 0) {
#pragma unroll
            for (int k = 0; k < NC; k++) {
                uint32_t* a = &csum[k][0][0];
                const uint32_t cv = lane < QI * (LT / 32) ? a[lane] : 0u;
                uint32_t x = cv;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (lane < QI * (LT / 32)) a[lane] = x - cv;
            }
        }
        __syncthreads();
        uint32_t run[NC];
        run[0] = v.tilecnt[tile];
        if (PAR) run[1] = opt.tiledrop[c0 + tile];
        if (SWP) run[NC - 1] = fin ? opt.tileswap[c0 + tile] : 0;
#pragma unroll
        for (int j = 0; j < QI; j++) {
            const int64_t t = 4 * (tile * (LTILE / 4) + (int64_t)j * LT + threadIdx.x);
            if (t >= nc) continue;
            int64_t b, c;
            bool first;
            decode(tp, v.sidx, lc, t, b, c, first);
            // entries of each counter before candidate t + i
            int64_t before[NC];
#pragma unroll
            for (int k = 0; k < NC; k++) before[k] = (int64_t)run[k] + csum[k][j][w] + pre[k][j];
            const int32_t gb = (int32_t)(base + b);
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t f = fw[j] >> (8 * i) & 0xffu;
                const int64_t wpre = before[0];
                const int64_t dpre = PAR ? before[1] : 0;
                const int64_t xpre = SWP ? before[NC - 1] : 0;
                const int64_t spre = t + i - wpre - dpre - xpre;  // strong entries before t + i
                if (i == 0 && first) {
                    v.woff[base + b] = (int32_t)min(W0 + wpre, (int64_t)INT32_MAX);
                    v.soff[base + b] = (int32_t)min(S0 + spre, (int64_t)INT32_MAX);
                    if (fin) xoff[base + b] = (int32_t)min(xpre, (int64_t)INT32_MAX);
                }
                if (PAR && f == 3) {
                    // a sibling covered by its parent's entry
                } else if (SWP && f >= 4) {
                    if (xpre < v.scap) {
                        xidx[xpre] = f == 5 ? (int32_t)(c + i) | SWAP_M2P : (int32_t)(c + i);
                        xtgt[xpre] = gb;
                    }
                } else if (f) {
                    const int64_t pos = W0 + wpre;
                    if (pos < v.wcap) {
                        v.widx[pos] = f == 2 ? (int32_t)(c >> 2) | PARENT_FLAG : (int32_t)(c + i);
                        if ((pos & 7) == 0) v.wrow[pos >> 3] = gb;
                    }
                } else {
                    const int64_t pos = S0 + spre;
                    if (pos < v.scap) {
                        v.sidx[pos] = (int32_t)(c + i);
                        v.stgt[pos] = gb;
                    }
                }
#pragma unroll
                for (int k = 0; k < NC; k++) before[k] += flag_in(f, k == 0 ? 0 : (PAR && k == 1) ? 1 : 2);
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
