// Structural checks of a tree and its lists: every invariant the evaluation kernels index by,
// tested with in-range reads only, so that a corrupted structure (for instance imported lists)
// is reported instead of being read out of bounds.  Violations set bits of a device word that
// the host turns into one error message.
#include <cmath>

#include "common.cuh"

namespace fmm {
namespace {

enum : int32_t {
    V_LEAF_BEGIN = 1,  // leaf offsets not 0 .. n, non-decreasing
    V_PERM = 2,        // the canonical order is not a permutation
    V_CLEAF = 4,       // a point's leaf disagrees with the leaf offsets
    V_RECTS = 8,       // a rectangle or radius not finite, or empty the wrong way round
    V_OFFSETS = 16,    // list offsets not 0 .. count, non-decreasing, or beyond the capacity
    V_WEAK = 32,       // a weak entry out of its level's range, or listed under another box
    V_STRONG = 64,     // the same for a strong entry
    V_EXCHANGE = 128,  // the same for the exchange lists
};

const char* const kVNames[] = {"leaf offsets", "canonical order (not a permutation)", "leaf of a point",
                               "box rectangles or radii", "list offsets", "weak-list entries",
                               "strong-list entries", "exchange-list entries"};

__device__ __forceinline__ int level_of(int64_t g) { return (63 - __clzll((unsigned long long)(3 * g + 1))) >> 1; }

// schedule: points (grid-stride over the instance's leaves, points and boxes)
__global__ void k_val_tree(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ lb,
                           const int32_t* __restrict__ perm, const int32_t* __restrict__ cleaf,
                           const double* __restrict__ rects, const double* __restrict__ rad,
                           int32_t* __restrict__ seen, int32_t* word)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    lb += S.lb0;
    perm += S.p0;
    cleaf += S.p0;
    seen += S.p0;
    rects += 4 * S.b0;
    rad += S.b0;
    const int64_t nleaf = level_size(S.L), n = S.n;
    const int64_t i0 = (int64_t)z.rank * blockDim.x + threadIdx.x, di = (int64_t)z.nb * blockDim.x;
    int32_t bad = 0;
    for (int64_t c = i0; c <= nleaf; c += di) {
        const int32_t v = lb[c];
        if ((c == 0 && v != 0) || (c == nleaf && v != n) || v < 0 || v > n || (c < nleaf && lb[c + 1] < v))
            bad |= V_LEAF_BEGIN;
    }
    for (int64_t i = i0; i < n; i += di) {
        const int32_t p = perm[i];
        if (p < 0 || p >= n) bad |= V_PERM;
        else atomicAdd(&seen[p], 1);
        const int32_t c = cleaf[i];
        if (c < 0 || c >= nleaf) {
            bad |= V_CLEAF;
        } else {
            const int32_t a = lb[c], b = lb[c + 1];
            if (i < a || i >= b) bad |= V_CLEAF;
        }
    }
    for (int64_t g = i0; g < S.nbox; g += di) {
        const double* r = rects + 4 * g;
        const bool fin = isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]) && isfinite(r[3]);
        if (!fin || !(r[0] <= r[1]) || !(r[2] <= r[3]) || !(rad[g] >= 0.0) || !isfinite(rad[g])) bad |= V_RECTS;
    }
    if (bad) atomicOr(word, bad);
}

// every input index exactly once; schedule: points
__global__ void k_val_perm(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ seen, int32_t* word)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    seen += S.p0;
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x)
        if (seen[i] != 1) {
            atomicOr(word, V_PERM);
            return;
        }
}

// offsets 0 .. count, non-decreasing, count within the capacity; schedule: points (boxes)
__device__ __forceinline__ bool offsets_bad(const int32_t* off, int64_t g, int64_t nbox, int64_t cap)
{
    const int32_t v = off[g];
    if (v < 0 || (g == 0 && v != 0) || (g < nbox && off[g + 1] < v)) return true;
    return g == nbox && (int64_t)v > cap;
}

__global__ void k_val_offsets(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                              const int32_t* __restrict__ woff, const int32_t* __restrict__ soff,
                              const int32_t* __restrict__ xoff, int32_t* word)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst T = LIs[z.i];
    woff += S.o0;
    soff += S.o0;
    const int64_t base = level_base(S.L);
    int32_t bad = 0;
    for (int64_t g = (int64_t)z.rank * blockDim.x + threadIdx.x; g <= S.nbox; g += (int64_t)z.nb * blockDim.x) {
        if (offsets_bad(woff, g, S.nbox, T.wcap) || offsets_bad(soff, g, S.nbox, T.scap)) bad |= V_OFFSETS;
        if (xoff) {  // exchange lists: empty below the finest level
            const int32_t* xo = xoff + S.o0;
            if (offsets_bad(xo, g, S.nbox, T.scap) || (g <= base && xo[g] != 0)) bad |= V_EXCHANGE;
        }
    }
    if (bad) atomicOr(word, bad);
}

// Entries: target within the instance and listed under it, source within its level (weak: or a
// parent entry of the level above; strong: within the level; exchange: a leaf).  Offsets are
// checked by k_val_offsets first; entries beyond the capacity are not read.  schedule: points
__global__ void k_val_entries(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                              const int32_t* __restrict__ woff, const int32_t* __restrict__ widx,
                              const int32_t* __restrict__ wrow, const int32_t* __restrict__ soff,
                              const int32_t* __restrict__ sidx, const int32_t* __restrict__ stgt,
                              const int32_t* __restrict__ xoff, const int32_t* __restrict__ xidx,
                              const int32_t* __restrict__ xtgt, const int32_t* word_in, int32_t* word)
{
    if (*word_in & V_OFFSETS) return;  // offsets are not trustworthy: entries are not looked at
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst T = LIs[z.i];
    woff += S.o0;
    soff += S.o0;
    widx += T.w0;
    wrow += T.w0 >> 3;
    sidx += T.s0;
    stgt += T.s0;
    const int64_t i0 = (int64_t)z.rank * blockDim.x + threadIdx.x, di = (int64_t)z.nb * blockDim.x;
    int32_t bad = 0;
    const int64_t nw = min((int64_t)woff[S.nbox], T.wcap), ns = min((int64_t)soff[S.nbox], T.scap);
    for (int64_t e = i0; e < nw; e += di) {
        // the target from the offsets (largest g with woff[g] <= e); every eighth entry's target
        // in the row table must agree, since the M2L kernels start their walks there
        int64_t lo = 0, hi = S.nbox;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (woff[mid] <= e) lo = mid;
            else hi = mid;
        }
        const int64_t g = lo;
        if (g < 1 || g >= S.nbox || ((e & 7) == 0 && wrow[e >> 3] != g)) {
            bad |= V_WEAK;
            continue;
        }
        const int l = level_of(g);
        const int32_t v = widx[e];
        const int32_t k = v & ~PARENT_FLAG;
        const bool ok = (v & PARENT_FLAG) ? (k >= 0 && k < level_size(l - 1)) : (v >= 0 && v < level_size(l));
        if (!ok) bad |= V_WEAK;
    }
    for (int64_t e = i0; e < ns; e += di) {
        const int64_t g = stgt[e];
        if (g < 0 || g >= S.nbox || e < soff[g] || e >= soff[g + 1]) {
            bad |= V_STRONG;
            continue;
        }
        const int32_t v = sidx[e];
        if (v < 0 || v >= level_size(level_of(g))) bad |= V_STRONG;
    }
    if (xoff && !(*word_in & V_EXCHANGE)) {
        const int32_t* xo = xoff + S.o0;
        xidx += T.s0;
        xtgt += T.s0;
        const int64_t nx = min((int64_t)xo[S.nbox], T.scap), base = level_base(S.L);
        for (int64_t e = i0; e < nx; e += di) {
            const int64_t g = xtgt[e];
            if (g < base || g >= S.nbox || e < xo[g] || e >= xo[g + 1]) {
                bad |= V_EXCHANGE;
                continue;
            }
            const int32_t v = xidx[e] & ~SWAP_M2P;
            if (v < 0 || v >= level_size(S.L)) bad |= V_EXCHANGE;
        }
    }
    if (bad) atomicOr(word, bad);
}

// targets of imported entries from the offsets; schedule: points (boxes)
__global__ void k_fill_targets(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs, int only,
                               const int32_t* __restrict__ woff, int32_t* __restrict__ wrow,
                               const int32_t* __restrict__ soff, int32_t* __restrict__ stgt)
{
    const Slot z = slot_of(sc);
    if (z.i != only) return;
    const Inst S = I[z.i];
    const LInst T = LIs[z.i];
    woff += S.o0;
    soff += S.o0;
    wrow += T.w0 >> 3;
    stgt += T.s0;
    // imported offsets are not trusted yet: every write stays within [0, capacity)
    for (int64_t g = (int64_t)z.rank * blockDim.x + threadIdx.x; g < S.nbox; g += (int64_t)z.nb * blockDim.x) {
        const int64_t w1 = min((int64_t)woff[g + 1], T.wcap), s1 = min((int64_t)soff[g + 1], T.scap);
        for (int64_t e = (max((int64_t)woff[g], (int64_t)0) + 7) & ~int64_t(7); e < w1; e += 8) wrow[e >> 3] = (int32_t)g;
        for (int64_t e = max((int64_t)soff[g], (int64_t)0); e < s1; e++) stgt[e] = (int32_t)g;
    }
}

}  // namespace

int validate(fmm_tree t, fmm_lists l, cudaStream_t s)
{
    int32_t* word = nullptr;
    int32_t* seen = t->segs;  // tree-build scratch, free outside builds
    if (cudaMalloc((void**)&word, 8) != cudaSuccess) return fail(FMM_ERR_OOM, "validation word");
    int rc = 0;
    auto body = [&]() -> int {
        FMM_CUDA(cudaMemsetAsync(word, 0, 8, s));
        FMM_CUDA(cudaMemsetAsync(seen, 0, 4 * (size_t)t->n, s));
        const unsigned gp = (unsigned)t->s_pts.blocks;
        const Sched sp = t->s_pts.d;
        k_val_tree<<<gp, 256, 0, s>>>(sp, t->dinst, t->leaf_begin, t->perm, t->cleaf, t->rects, t->radii, seen, word);
        note_launch();
        k_val_perm<<<gp, 256, 0, s>>>(sp, t->dinst, seen, word); note_launch();
        if (l) {
            const bool x = (l->mode & FMM_LISTS_EXCHANGE) != 0;
            k_val_offsets<<<gp, 256, 0, s>>>(sp, t->dinst, l->dlinst, l->woff, l->soff, x ? l->xoff : nullptr, word);
            note_launch();
            // the entry check reads the offsets' verdict from a copy made after k_val_offsets
            FMM_CUDA(cudaMemcpyAsync(word + 1, word, 4, cudaMemcpyDeviceToDevice, s));
            k_val_entries<<<gp, 256, 0, s>>>(sp, t->dinst, l->dlinst, l->woff, l->widx, l->wrow, l->soff, l->sidx,
                                             l->stgt, x ? l->xoff : nullptr, l->xidx, l->xtgt, word + 1, word);
            note_launch();
        }
        FMM_LAUNCH_CHECK("validate");
        FMM_CUDA(cudaStreamSynchronize(s));
        int32_t w = 0;
        FMM_CUDA(cudaMemcpy(&w, word, 4, cudaMemcpyDeviceToHost));
        for (int b = 0; b < 8; b++)
            if (w & (1 << b)) return fail(FMM_ERR_STATE, "validation failed: %s", kVNames[b]);
        return FMM_OK;
    };
    rc = body();
    cudaFree(word);
    return rc;
}

int lists_import(fmm_lists l, int i, const int32_t* woff, const int32_t* widx, const int32_t* soff,
                 const int32_t* sidx, cudaStream_t s)
{
    fmm_tree t = l->tree;
    const Inst& S = t->hinst[i];
    const LInst& T = l->hlinst[i];
    int32_t nw = 0, ns = 0;
    FMM_CUDA(cudaStreamSynchronize(s));
    FMM_CUDA(cudaMemcpy(&nw, woff + S.nbox, 4, cudaMemcpyDeviceToHost));
    FMM_CUDA(cudaMemcpy(&ns, soff + S.nbox, 4, cudaMemcpyDeviceToHost));
    if (nw < 0 || ns < 0 || (int64_t)nw > T.wcap || (int64_t)ns > T.scap)
        return fail(FMM_ERR_CAPACITY, "instance %d: %d weak / %d strong entries, capacity %lld / %lld", i, nw, ns,
                    (long long)T.wcap, (long long)T.scap);
    FMM_CUDA(cudaMemcpyAsync(l->woff + S.o0, woff, 4 * (S.nbox + 1), cudaMemcpyDeviceToDevice, s));
    FMM_CUDA(cudaMemcpyAsync(l->soff + S.o0, soff, 4 * (S.nbox + 1), cudaMemcpyDeviceToDevice, s));
    if (nw) FMM_CUDA(cudaMemcpyAsync(l->widx + T.w0, widx, 4 * (size_t)nw, cudaMemcpyDeviceToDevice, s));
    if (ns) FMM_CUDA(cudaMemcpyAsync(l->sidx + T.s0, sidx, 4 * (size_t)ns, cudaMemcpyDeviceToDevice, s));
    k_fill_targets<<<(unsigned)t->s_pts.blocks, 256, 0, s>>>(t->s_pts.d, t->dinst, l->dlinst, i, l->woff, l->wrow,
                                                             l->soff, l->stgt);
    note_launch();
    FMM_LAUNCH_CHECK("lists import");
    return 0;
}

}  // namespace fmm
