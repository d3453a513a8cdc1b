// Launch schedules of forests: how the blocks of one launch are shared out over the instances.
//
// Every kernel that covers all instances of a forest runs on a 1-D grid and finds its instance,
// its rank among that instance's blocks and their number from two small tables (struct Sched).
// The tables are built here, on the host, from quantities known when the tree is created (point
// and box counts, levels) and copied to the device once; launches then need no host work.  The
// per-instance block counts follow the work of each kernel family:
//   tiles     one block per tree-build tile (exact)
//   local     one block per box of the level where the median tree finishes inside blocks
//   points    one block per 1024 points
//   levels    one block per 4 boxes (warp-per-box kernels) or per 128 boxes (thread-per-box)
//   lists     one block per tile of about 9 * 4^l candidates of level l
//   M2L       a total budget shared in proportion to the boxes (weak pairs grow with them)
//   near      a total budget shared in proportion to n * (largest leaf): the pair evaluations
// A forest of one instance keeps no tables: its blocks are the whole grid.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "common.cuh"

namespace fmm {

namespace {

constexpr int64_t PTS_PER_BLOCK = 1024;
constexpr int64_t LIST_TILE = 2048;        // candidates per tile of the list kernels
constexpr int DEFAULT_M2L_BLOCKS = 152 * 16;
constexpr int DEFAULT_P2P_BLOCKS = 152 * 8;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

int make_from(fmm_tree t, const std::vector<int64_t>& b, SchedH& out)
{
    sched_free(out);
    return sched_make(t, b.data(), out);
}

// A budget of `total` blocks shared in proportion to the weights (at least one block for every
// instance of positive weight).
std::vector<int64_t> share(const std::vector<double>& w, int64_t total)
{
    double W = 0;
    for (double v : w) W += v;
    std::vector<int64_t> b(w.size(), 0);
    for (size_t i = 0; i < w.size(); i++)
        if (w[i] > 0) b[i] = std::max<int64_t>(1, (int64_t)std::llround((double)total * w[i] / W));
    return b;
}

}  // namespace

void sched_free(SchedH& h)
{
    if (h.mem) cudaFree(h.mem);
    h = SchedH{};
}

int sched_make(fmm_tree t, const int64_t* blocks, SchedH& out)
{
    out = SchedH{};
    const int ni = t->n_inst;
    int64_t total = 0;
    for (int i = 0; i < ni; i++) total += std::max<int64_t>(0, blocks[i]);
    if (total >= INT32_MAX) return fail(FMM_ERR_ARG, "launch of %lld blocks is too large", (long long)total);
    out.blocks = (int)total;
    if (ni == 1 || total == 0) return 0;
    const int64_t inst_words = (total + 1) & ~int64_t(1);  // keep the span table 8-byte aligned
    std::vector<int32_t> h(inst_words + 2 * (size_t)ni, 0);
    int64_t b = 0;
    for (int i = 0; i < ni; i++) {
        const int64_t c = std::max<int64_t>(0, blocks[i]);
        h[inst_words + 2 * i] = (int32_t)b;
        h[inst_words + 2 * i + 1] = (int32_t)c;
        for (int64_t k = 0; k < c; k++) h[b + k] = i;
        b += c;
    }
    void* mem = nullptr;
    if (cudaMalloc(&mem, 4 * h.size()) != cudaSuccess) return fail(FMM_ERR_OOM, "launch schedule");
    cudaError_t e = cudaMemcpy(mem, h.data(), 4 * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return cuda_fail(e, "launch schedule upload");
    }
    out.mem = mem;
    out.d.inst = (const int32_t*)mem;
    out.d.span = (const int2*)((const int32_t*)mem + inst_words);
    return 0;
}

int sched_all(fmm_tree t)
{
    const int ni = t->n_inst, Lm = t->Lmax;
    std::vector<int64_t> b(ni);
    int rc;
    auto each = [&](auto f) {
        for (int i = 0; i < ni; i++) b[i] = f(t->hinst[i]);
    };
    each([](const Inst& S) { return S.ntiles; });
    if ((rc = make_from(t, b, t->s_tiles))) return rc;
    each([](const Inst& S) { return cdiv(S.n, PTS_PER_BLOCK); });
    if ((rc = make_from(t, b, t->s_pts))) return rc;
    each([](const Inst& S) { return cdiv(256, rs_digits_per_block(S.ntiles)); });
    if ((rc = make_from(t, b, t->s_rsscan))) return rc;
    each([](const Inst& S) { return S.L >= 1 ? cdiv(level_size(S.L), 4) : 0; });
    if ((rc = make_from(t, b, t->s_p2m))) return rc;
    t->s_split = new (std::nothrow) SchedH[std::max(Lm, 1)];
    t->s_m2m = new (std::nothrow) SchedH[std::max(Lm, 1)];
    t->s_l2l = new (std::nothrow) SchedH[std::max(Lm, 1)];
    t->s_lists = new (std::nothrow) SchedH[Lm + 1];
    if (!t->s_split || !t->s_m2m || !t->s_l2l || !t->s_lists) return fail(FMM_ERR_OOM, "host allocation");
    each([](const Inst& S) { return S.lg < S.L ? level_size(S.lg) : 0; });
    if ((rc = make_from(t, b, t->s_local))) return rc;
    for (int l = 0; l < Lm; l++) {
        each([l](const Inst& S) { return l < S.lg ? cdiv(level_size(l), 128) : 0; });
        if ((rc = make_from(t, b, t->s_split[l]))) return rc;
        each([l](const Inst& S) { return l >= 1 && l < S.L ? cdiv(level_size(l), 4) : 0; });
        if ((rc = make_from(t, b, t->s_m2m[l]))) return rc;
        each([l](const Inst& S) { return l >= 1 && l < S.L ? cdiv(level_size(l + 1), 4) : 0; });
        if ((rc = make_from(t, b, t->s_l2l[l]))) return rc;
    }
    for (int l = 0; l <= Lm; l++) {
        each([l](const Inst& S) { return l >= 1 && l <= S.L ? cdiv(9 * level_size(l), LIST_TILE) : 0; });
        if ((rc = make_from(t, b, t->s_lists[l]))) return rc;
    }
    return sched_tuned(t);
}

int sched_tuned(fmm_tree t)
{
    const int ni = t->n_inst;
    std::vector<double> wm(ni), wp(ni);
    for (int i = 0; i < ni; i++) {
        const Inst& S = t->hinst[i];
        const int64_t leaf = (S.n + level_size(S.L) - 1) / level_size(S.L);
        wm[i] = S.L >= 1 ? (double)S.nbox : 0.0;
        wp[i] = (double)S.n * (double)leaf;
    }
    const int m2l = t->tune_m2l_blocks > 0 ? t->tune_m2l_blocks : DEFAULT_M2L_BLOCKS;
    const int p2p = t->tune_p2p_blocks > 0 ? t->tune_p2p_blocks : DEFAULT_P2P_BLOCKS;
    int rc;
    if ((rc = make_from(t, share(wm, m2l), t->s_m2l))) return rc;
    return make_from(t, share(wp, p2p), t->s_p2p);
}

void sched_free_all(fmm_tree t)
{
    sched_free(t->s_tiles);
    sched_free(t->s_pts);
    sched_free(t->s_rsscan);
    sched_free(t->s_p2m);
    sched_free(t->s_local);
    sched_free(t->s_m2l);
    sched_free(t->s_p2p);
    const int Lm = t->Lmax;
    if (t->s_split)
        for (int l = 0; l < std::max(Lm, 1); l++) sched_free(t->s_split[l]);
    if (t->s_m2m)
        for (int l = 0; l < std::max(Lm, 1); l++) sched_free(t->s_m2m[l]);
    if (t->s_l2l)
        for (int l = 0; l < std::max(Lm, 1); l++) sched_free(t->s_l2l[l]);
    if (t->s_lists)
        for (int l = 0; l <= Lm; l++) sched_free(t->s_lists[l]);
    delete[] t->s_split;
    delete[] t->s_m2m;
    delete[] t->s_l2l;
    delete[] t->s_lists;
    t->s_split = t->s_m2m = t->s_l2l = t->s_lists = nullptr;
}

}  // namespace fmm
