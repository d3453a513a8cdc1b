// The C ABI of libfmm_gb300.so (declared in include/fmm.h): argument checks, handle lifetime,
// device selection and the device status word.  All computation is in the kernels of tree.cu,
// lists.cu, scan.cu and expand.cu.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"

namespace fmm {

static thread_local char g_msg[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(FMM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

static std::atomic<int64_t> g_launches{0};
static std::mutex g_prof_mutex;
static bool g_prof_on = false;
struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};
static std::vector<ProfRec> g_prof_recs;
static std::vector<cudaEvent_t> g_prof_pool;
static cudaEvent_t g_prof_open[FMM_STAGE_COUNT] = {};

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void prof_mark(int stage, bool begin, cudaStream_t s)
{
    if (!g_prof_on || stage < 0 || stage >= FMM_STAGE_COUNT) return;
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    cudaEvent_t e;
    if (!g_prof_pool.empty()) {
        e = g_prof_pool.back();
        g_prof_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return;
    }
    cudaEventRecord(e, s);
    if (begin) {
        if (g_prof_open[stage]) g_prof_pool.push_back(g_prof_open[stage]);
        g_prof_open[stage] = e;
    } else if (g_prof_open[stage]) {
        g_prof_recs.push_back({stage, g_prof_open[stage], e});
        g_prof_open[stage] = nullptr;
    } else {
        g_prof_pool.push_back(e);
    }
}

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define GUARD(dev)                                                               \
    DeviceGuard guard_(dev);                                                     \
    if (!guard_.ok) return fail(FMM_ERR_CUDA, "cannot select device %d", (dev));

void free_tree(fmm_tree t)
{
    if (!t) return;
    void* ptrs[] = {t->lb_bal, t->rects, t->centers, t->radii, t->rad32, t->cen_hi, t->cen_lo, t->perm, t->leaf_begin,
                    t->leaf_of, t->xs, t->ys, t->dxf, t->dyf, t->keys, t->vals, t->rs_counts,
                    t->rs_totals, t->tilecnt, t->hflag, t->bbox_keys, t->ones_before, t->node_off, t->segs, t->status,
                    t->Me, t->Le, t->Mf, t->Lf, t->pk64, t->pk32, t->acc, t->acc32, t->cleaf, t->dinst, t->Lf0lo,
                    t->pkf, t->qf, t->accf, t->qmem, t->pkff, t->mff};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    sched_free_all(t);
    for (cudaEvent_t e : t->ev)
        if (e) cudaEventDestroy(e);
    if (t->ev_level) {
        for (int i = 0; i <= t->Lmax; i++)
            if (t->ev_level[i]) cudaEventDestroy(t->ev_level[i]);
        delete[] t->ev_level;
    }
    if (t->side) cudaStreamDestroy(t->side);
    if (t->own_hinst) delete[] t->hinst;
    delete t;
}

void free_lists(fmm_lists l)
{
    if (!l) return;
    void* ptrs[] = {l->woff, l->soff, l->widx, l->wrow, l->rowtgt, l->sidx, l->stgt, l->flags, l->tilecnt, l->status,
                    l->dlinst, l->tiledrop, l->tileswap, l->xoff, l->xidx, l->xtgt, l->p2p_items, l->p2p_pos,
                    l->p2p_tmp, l->p2p_zero};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete[] l->hlinst;
    delete l;
}

int status_to_code(int32_t st)
{
    if (st & ST_NONFINITE) return fail(FMM_ERR_NONFINITE, "non-finite coordinate or strength");
    if (st & ST_CAPACITY) return fail(FMM_ERR_CAPACITY, "interaction lists exceed the capacity");
    if (st & ST_TIMEOUT) return fail(FMM_ERR_TIMEOUT, "a bounded device wait gave up");
    if (st & ST_DEGENERATE)
        return fail(FMM_ERR_DEGENERATE, "a leaf box of zero size: the far part of the field is undefined there");
    if (st & ST_ARG) return fail(FMM_ERR_STATE, "inconsistent internal state detected on the device");
    return FMM_OK;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" {

const char* fmm_last_error(void) { return g_msg; }

int fmm_profile_enable(int on)
{
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    g_prof_on = on != 0;
    return FMM_OK;
}

int fmm_profile_read(double* ms, int64_t* count, int nstages)
{
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    int nread = 0;
    for (const ProfRec& r : g_prof_recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
            return fail(FMM_ERR_CUDA, "profile events");
        if (r.stage < nstages) {
            if (ms) ms[r.stage] += t;
            if (count) count[r.stage] += 1;
        }
        g_prof_pool.push_back(r.a);
        g_prof_pool.push_back(r.b);
        nread++;
    }
    g_prof_recs.clear();
    return nread;
}

int64_t fmm_launch_count(void) { return g_launches.load(); }

int fmm_tree_create_batched(int n_inst, const int64_t* n, const int* levels, fmm_tree* out)
{
    if (!out || !n || !levels) return fail(FMM_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (n_inst < 1 || n_inst > FMM_MAX_INSTANCES)
        return fail(FMM_ERR_ARG, "n_inst = %d outside [1, %d]", n_inst, FMM_MAX_INSTANCES);
    int64_t total = 0;
    for (int i = 0; i < n_inst; i++) {
        if (levels[i] < 0 || levels[i] > 13)
            return fail(FMM_ERR_ARG, "instance %d: levels = %d outside [0, 13]", i, levels[i]);
        if (n[i] < 1 || n[i] >= ((int64_t)1 << 31) - 1)
            return fail(FMM_ERR_ARG, "instance %d: n = %lld outside [1, 2^31)", i, (long long)n[i]);
        if (n[i] < level_size(levels[i]))
            return fail(FMM_ERR_LEVELS, "instance %d: n = %lld < 4^%d: some leaf would be empty", i,
                        (long long)n[i], levels[i]);
        total += n[i];
    }
    if (total >= ((int64_t)1 << 31) - 1)
        return fail(FMM_ERR_ARG, "total of %lld points is not below 2^31 - 1", (long long)total);
    fmm_tree t = new (std::nothrow) fmm_tree_s();
    if (!t) return fail(FMM_ERR_OOM, "host allocation");
    if (cudaGetDevice(&t->dev) != cudaSuccess) {
        delete t;
        return fail(FMM_ERR_CUDA, "no CUDA device");
    }
    int rc;
    try {
        rc = tree_alloc(t, n_inst, n, levels);
    } catch (...) {
        rc = fail(FMM_ERR_OOM, "host allocation");
    }
    if (rc) {
        free_tree(t);
        return rc;
    }
    *out = t;
    return FMM_OK;
}

int fmm_tree_create(int64_t n, int levels, fmm_tree* out)
{
    return fmm_tree_create_batched(1, &n, &levels, out);
}

int fmm_build_tree(fmm_tree t, const double* x, const double* y, void* stream)
{
    if (!t || !x || !y) return fail(FMM_ERR_ARG, "NULL argument");
    GUARD(t->dev);
    return tree_build(t, x, y, (cudaStream_t)stream);
}

int fmm_build_tree_uniform(fmm_tree t, const double* x, const double* y, const double* root_host, void* stream)
{
    if (!t || !x || !y) return fail(FMM_ERR_ARG, "NULL argument");
    if (root_host && !(root_host[2] >= 0.0 && std::isfinite(root_host[0]) && std::isfinite(root_host[1]) &&
                       std::isfinite(root_host[2])))
        return fail(FMM_ERR_ARG, "the root square needs finite x0, y0 and a side >= 0");
    GUARD(t->dev);
    return tree_build_uniform(t, x, y, root_host, (cudaStream_t)stream);
}

int fmm_tree_export(fmm_tree t, int32_t* perm, double* rects, int32_t* leaf_begin, void* stream)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (!t->built) return fail(FMM_ERR_STATE, "tree not built");
    GUARD(t->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (perm) FMM_CUDA(cudaMemcpyAsync(perm, t->perm, 4 * t->n, cudaMemcpyDeviceToDevice, s));
    if (rects) FMM_CUDA(cudaMemcpyAsync(rects, t->rects, 32 * t->nbox, cudaMemcpyDeviceToDevice, s));
    if (leaf_begin)
        FMM_CUDA(cudaMemcpyAsync(leaf_begin, t->leaf_begin, 4 * (t->nleaf + t->n_inst), cudaMemcpyDeviceToDevice, s));
    return FMM_OK;
}

int fmm_tree_info(fmm_tree t, int64_t* n, int* levels, int64_t* nbox)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (n) *n = t->n;
    if (levels) *levels = t->Lmax;
    if (nbox) *nbox = t->nbox;
    return FMM_OK;
}

int fmm_tree_num_instances(fmm_tree t)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    return t->n_inst;
}

int fmm_tree_instance(fmm_tree t, int i, int64_t* p0, int64_t* n, int* levels, int64_t* b0, int64_t* nbox,
                      int64_t* lb0)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (i < 0 || i >= t->n_inst) return fail(FMM_ERR_ARG, "instance %d outside [0, %d)", i, t->n_inst);
    const Inst& S = t->hinst[i];
    if (p0) *p0 = S.p0;
    if (n) *n = S.n;
    if (levels) *levels = S.L;
    if (b0) *b0 = S.b0;
    if (nbox) *nbox = S.nbox;
    if (lb0) *lb0 = S.lb0;
    return FMM_OK;
}

void fmm_tree_destroy(fmm_tree t)
{
    if (!t) return;
    DeviceGuard g(t->dev);
    free_tree(t);
}

namespace {

int lists_create_impl(fmm_tree t, const int64_t* wcap, const int64_t* scap, fmm_lists* out)
{
    fmm_lists l = new (std::nothrow) fmm_lists_s();
    if (!l) return fail(FMM_ERR_OOM, "host allocation");
    l->tree = t;
    int rc;
    try {
        rc = lists_alloc(t, l, wcap, scap);
    } catch (...) {
        rc = fail(FMM_ERR_OOM, "host allocation");
    }
    if (rc) {
        free_lists(l);
        return rc;
    }
    *out = l;
    return FMM_OK;
}

}  // namespace

int fmm_lists_create(fmm_tree t, int64_t weak_capacity, int64_t strong_capacity, fmm_lists* out)
{
    if (!t || !out) return fail(FMM_ERR_ARG, "NULL argument");
    *out = nullptr;
    GUARD(t->dev);
    if (weak_capacity >= INT32_MAX || strong_capacity >= INT32_MAX)
        return fail(FMM_ERR_ARG, "capacity must be below 2^31 - 1");
    // one instance: the capacities as given; several: shared out in proportion to the box counts
    std::vector<int64_t> w(t->n_inst), st(t->n_inst);
    for (int i = 0; i < t->n_inst; i++) {
        const Inst& S = t->hinst[i];
        const double share = (double)S.nbox / (double)t->nbox;
        w[i] = weak_capacity <= 0 ? 64 * S.nbox
               : t->n_inst == 1   ? weak_capacity
                                  : std::max<int64_t>(16 * S.nbox, (int64_t)(share * (double)weak_capacity));
        st[i] = strong_capacity <= 0 ? 32 * S.nbox
                : t->n_inst == 1     ? strong_capacity
                                     : std::max<int64_t>(8 * S.nbox, (int64_t)(share * (double)strong_capacity));
    }
    return lists_create_impl(t, w.data(), st.data(), out);
}

int fmm_lists_create_batched(fmm_tree t, const int64_t* weak_capacity, const int64_t* strong_capacity,
                             fmm_lists* out)
{
    if (!t || !out || !weak_capacity || !strong_capacity) return fail(FMM_ERR_ARG, "NULL argument");
    *out = nullptr;
    GUARD(t->dev);
    for (int i = 0; i < t->n_inst; i++)
        if (weak_capacity[i] < 1 || strong_capacity[i] < 1)
            return fail(FMM_ERR_ARG, "instance %d: capacities must be positive", i);
    return lists_create_impl(t, weak_capacity, strong_capacity, out);
}

int fmm_lists_set_mode(fmm_lists l, int mode)
{
    if (!l) return fail(FMM_ERR_ARG, "NULL lists");
    if (mode & ~(FMM_LISTS_PARENTS | FMM_LISTS_EXCHANGE)) return fail(FMM_ERR_ARG, "unknown lists mode %d", mode);
    GUARD(l->tree->dev);
    int64_t words = 0, scap = 0;
    for (int i = 0; i < l->tree->n_inst; i++) {
        words += lists_tile_words(l->hlinst[i].scap);
        scap += l->hlinst[i].scap;
    }
    if ((mode & FMM_LISTS_PARENTS) && !l->tiledrop &&
        cudaMalloc((void**)&l->tiledrop, 4 * words) != cudaSuccess)
        return fail(FMM_ERR_OOM, "list storage");
    if ((mode & FMM_LISTS_EXCHANGE) && !l->tileswap) {
        if (cudaMalloc((void**)&l->tileswap, 4 * words) != cudaSuccess ||
            cudaMalloc((void**)&l->xoff, 4 * (size_t)(l->tree->nbox + l->tree->n_inst)) != cudaSuccess ||
            cudaMalloc((void**)&l->xidx, 4 * (size_t)std::max<int64_t>(scap, 1)) != cudaSuccess ||
            cudaMalloc((void**)&l->xtgt, 4 * (size_t)std::max<int64_t>(scap, 1)) != cudaSuccess)
            return fail(FMM_ERR_OOM, "list storage");
    }
    l->mode = mode;
    l->built = false;  // the lists must be rebuilt in the new mode
    return FMM_OK;
}

int fmm_lists_export_exchange(fmm_lists l, int i, int32_t* xoff, int32_t* xidx, int64_t* count, void* stream)
{
    if (!l) return fail(FMM_ERR_ARG, "NULL lists");
    if (!l->built) return fail(FMM_ERR_STATE, "lists not built");
    if (!(l->mode & FMM_LISTS_EXCHANGE)) return fail(FMM_ERR_STATE, "the lists were built without the role exchange");
    fmm_tree t = l->tree;
    if (i < 0 || i >= t->n_inst) return fail(FMM_ERR_ARG, "instance %d outside [0, %d)", i, t->n_inst);
    GUARD(t->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const Inst& S = t->hinst[i];
    const LInst& T = l->hlinst[i];
    FMM_CUDA(cudaStreamSynchronize(s));
    int32_t x = 0;
    FMM_CUDA(cudaMemcpy(&x, l->xoff + S.o0 + S.nbox, 4, cudaMemcpyDeviceToHost));
    if (count) *count = x;
    if (xoff) FMM_CUDA(cudaMemcpyAsync(xoff, l->xoff + S.o0, 4 * (S.nbox + 1), cudaMemcpyDeviceToDevice, s));
    if (xidx && x > 0)
        FMM_CUDA(cudaMemcpyAsync(xidx, l->xidx + T.s0, 4 * std::min<int64_t>(x, T.scap), cudaMemcpyDeviceToDevice, s));
    FMM_CUDA(cudaStreamSynchronize(s));
    return FMM_OK;
}

int fmm_interaction_lists(fmm_tree t, fmm_lists l, double theta, void* stream)
{
    if (!t || !l) return fail(FMM_ERR_ARG, "NULL handle");
    if (l->tree != t) return fail(FMM_ERR_STATE, "lists were created for another tree");
    if (!t->built) return fail(FMM_ERR_STATE, "tree not built");
    if (!(theta > 0.0 && theta < 1.0)) return fail(FMM_ERR_ARG, "theta = %g outside (0, 1)", theta);
    GUARD(t->dev);
    return lists_build(t, l, theta, (cudaStream_t)stream);
}

namespace {

// Per-instance entry counts (ends of the CSR offsets) and the list status word.
int read_counts(fmm_lists l, cudaStream_t s, std::vector<int32_t>& woff, std::vector<int32_t>& soff,
                int32_t& st)
{
    fmm_tree t = l->tree;
    const int64_t m = t->nbox + t->n_inst;
    woff.resize(m);
    soff.resize(m);
    FMM_CUDA(cudaStreamSynchronize(s));
    FMM_CUDA(cudaMemcpy(woff.data(), l->woff, 4 * m, cudaMemcpyDeviceToHost));
    FMM_CUDA(cudaMemcpy(soff.data(), l->soff, 4 * m, cudaMemcpyDeviceToHost));
    FMM_CUDA(cudaMemcpy(&st, l->status, 4, cudaMemcpyDeviceToHost));
    return 0;
}

}  // namespace

int fmm_lists_counts(fmm_lists l, void* stream, int64_t* n_weak, int64_t* n_strong)
{
    if (!l) return fail(FMM_ERR_ARG, "NULL lists");
    if (!l->built) return fail(FMM_ERR_STATE, "lists not built");
    GUARD(l->tree->dev);
    std::vector<int32_t> wo, so;
    int32_t st = 0;
    int rc = read_counts(l, (cudaStream_t)stream, wo, so, st);
    if (rc) return rc;
    fmm_tree t = l->tree;
    int bad = -1;
    for (int i = 0; i < t->n_inst; i++) {
        const Inst& S = t->hinst[i];
        const LInst& T = l->hlinst[i];
        const int64_t w = wo[S.o0 + S.nbox], sc = so[S.o0 + S.nbox];
        if (n_weak) n_weak[i] = w;
        if (n_strong) n_strong[i] = sc;
        if (bad < 0 && (w > T.wcap || sc > T.scap)) bad = i;
    }
    if (st & ST_CAPACITY) {
        if (bad < 0) bad = 0;
        const Inst& S = t->hinst[bad];
        return fail(FMM_ERR_CAPACITY, "instance %d: lists need %d weak / %d strong entries, capacity %lld / %lld",
                    bad, wo[S.o0 + S.nbox], so[S.o0 + S.nbox], (long long)l->hlinst[bad].wcap,
                    (long long)l->hlinst[bad].scap);
    }
    return FMM_OK;
}

int fmm_lists_sync(fmm_lists l, void* stream, int64_t* n_weak, int64_t* n_strong)
{
    if (!l) return fail(FMM_ERR_ARG, "NULL lists");
    if (!l->built) return fail(FMM_ERR_STATE, "lists not built");
    const int ni = l->tree->n_inst;
    std::vector<int64_t> w(ni), st(ni);
    const int rc = fmm_lists_counts(l, stream, w.data(), st.data());
    int64_t sw = 0, ss = 0;
    for (int i = 0; i < ni; i++) {
        sw += w[i];
        ss += st[i];
    }
    if (n_weak) *n_weak = sw;
    if (n_strong) *n_strong = ss;
    return rc;
}

int fmm_lists_export_instance(fmm_lists l, int i, int32_t* woff, int32_t* widx, int32_t* soff, int32_t* sidx,
                              void* stream)
{
    if (!l) return fail(FMM_ERR_ARG, "NULL lists");
    if (!l->built) return fail(FMM_ERR_STATE, "lists not built");
    fmm_tree t = l->tree;
    if (i < 0 || i >= t->n_inst) return fail(FMM_ERR_ARG, "instance %d outside [0, %d)", i, t->n_inst);
    GUARD(t->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const Inst& S = t->hinst[i];
    const LInst& T = l->hlinst[i];
    FMM_CUDA(cudaStreamSynchronize(s));
    int32_t w = 0, st = 0;
    FMM_CUDA(cudaMemcpy(&w, l->woff + S.o0 + S.nbox, 4, cudaMemcpyDeviceToHost));
    FMM_CUDA(cudaMemcpy(&st, l->soff + S.o0 + S.nbox, 4, cudaMemcpyDeviceToHost));
    const int64_t nb = S.nbox + 1;
    if (woff) FMM_CUDA(cudaMemcpyAsync(woff, l->woff + S.o0, 4 * nb, cudaMemcpyDeviceToDevice, s));
    if (soff) FMM_CUDA(cudaMemcpyAsync(soff, l->soff + S.o0, 4 * nb, cudaMemcpyDeviceToDevice, s));
    if (widx && w > 0)
        FMM_CUDA(cudaMemcpyAsync(widx, l->widx + T.w0, 4 * std::min<int64_t>(w, T.wcap), cudaMemcpyDeviceToDevice, s));
    if (sidx && st > 0)
        FMM_CUDA(cudaMemcpyAsync(sidx, l->sidx + T.s0, 4 * std::min<int64_t>(st, T.scap), cudaMemcpyDeviceToDevice, s));
    return FMM_OK;
}

int fmm_lists_export(fmm_lists l, int32_t* woff, int32_t* widx, int32_t* soff, int32_t* sidx, void* stream)
{
    if (!l) return fail(FMM_ERR_ARG, "NULL lists");
    if (l->tree->n_inst != 1)
        return fail(FMM_ERR_ARG, "the tree holds %d instances: use fmm_lists_export_instance", l->tree->n_inst);
    return fmm_lists_export_instance(l, 0, woff, widx, soff, sidx, stream);
}

int fmm_lists_import(fmm_lists l, int i, const int32_t* woff, const int32_t* widx, const int32_t* soff,
                     const int32_t* sidx, void* stream)
{
    if (!l || !woff || !soff) return fail(FMM_ERR_ARG, "NULL argument");
    fmm_tree t = l->tree;
    if (i < 0 || i >= t->n_inst) return fail(FMM_ERR_ARG, "instance %d outside [0, %d)", i, t->n_inst);
    if (!t->built) return fail(FMM_ERR_STATE, "tree not built");
    if (l->mode & FMM_LISTS_EXCHANGE) return fail(FMM_ERR_STATE, "lists with exchange lists cannot be imported");
    GUARD(t->dev);
    const int rc = lists_import(l, i, woff, widx, soff, sidx, (cudaStream_t)stream);
    if (rc) return rc;
    l->built = true;
    return FMM_OK;
}

int fmm_validate(fmm_tree t, fmm_lists l, void* stream)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (!t->built) return fail(FMM_ERR_STATE, "tree not built");
    if (l && l->tree != t) return fail(FMM_ERR_STATE, "lists were created for another tree");
    if (l && !l->built) return fail(FMM_ERR_STATE, "lists not built");
    GUARD(t->dev);
    return validate(t, l, (cudaStream_t)stream);
}

int fmm_selftest_bounded_wait(int64_t tries, void* stream)
{
    if (tries < 1 || tries > (int64_t(1) << 20)) return fail(FMM_ERR_ARG, "tries = %lld outside [1, 2^20]", (long long)tries);
    return bounded_wait_selftest(tries, (cudaStream_t)stream);
}

int fmm_selftest_queue_timeout(fmm_tree t, int64_t tries, void* stream)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (tries < 1 || tries > (int64_t(1) << 20)) return fail(FMM_ERR_ARG, "tries = %lld outside [1, 2^20]", (long long)tries);
    GUARD(t->dev);
    return queue_timeout_selftest(t, tries, (cudaStream_t)stream);
}

void fmm_lists_destroy(fmm_lists l)
{
    if (!l) return;
    DeviceGuard g(l->tree->dev);
    free_lists(l);
}

int fmm_evaluate(fmm_tree t, fmm_lists l, const double* q, const fmm_params* prm, double* phi, void* stream)
{
    if (!t || !l || !q || !prm || !phi) return fail(FMM_ERR_ARG, "NULL argument");
    if (l->tree != t) return fail(FMM_ERR_STATE, "lists were created for another tree");
    if (!t->built || !l->built) return fail(FMM_ERR_STATE, "tree or lists not built");
    if (prm->p < 0 || prm->p > 40) return fail(FMM_ERR_ARG, "p = %d outside [0, 40]", prm->p);
    if (prm->mode != FMM_MODE_FP64 && prm->mode != FMM_MODE_MIXED && prm->mode != FMM_MODE_SPLIT)
        return fail(FMM_ERR_ARG, "unknown mode %d", prm->mode);
    GUARD(t->dev);
    return evaluate(t, l, q, *prm, phi, (cudaStream_t)stream);
}

int fmm_step(fmm_tree t, fmm_lists l, const double* x, const double* y, double theta, const double* q,
             const fmm_params* prm, double* phi, void* stream)
{
    if (!t || !l || !x || !y || !q || !prm || !phi) return fail(FMM_ERR_ARG, "NULL argument");
    if (l->tree != t) return fail(FMM_ERR_STATE, "lists were created for another tree");
    if (!(theta > 0.0 && theta < 1.0)) return fail(FMM_ERR_ARG, "theta = %g outside (0, 1)", theta);
    if (prm->p < 0 || prm->p > 40) return fail(FMM_ERR_ARG, "p = %d outside [0, 40]", prm->p);
    if (prm->mode != FMM_MODE_FP64 && prm->mode != FMM_MODE_MIXED && prm->mode != FMM_MODE_SPLIT)
        return fail(FMM_ERR_ARG, "unknown mode %d", prm->mode);
    GUARD(t->dev);
    if (!t->side) {
        FMM_CUDA(cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking));
        for (cudaEvent_t& e : t->ev) FMM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        t->ev_level = new (std::nothrow) cudaEvent_t[t->Lmax + 1]();
        if (!t->ev_level) return fail(FMM_ERR_OOM, "host allocation");
        for (int i = 0; i <= t->Lmax; i++) FMM_CUDA(cudaEventCreateWithFlags(&t->ev_level[i], cudaEventDisableTiming));
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the lists of each level are built on the second stream as soon as the tree build has the
    // geometry of that level
    int rc = tree_build(t, x, y, s, t->ev_level);
    if (rc) return rc;
    rc = lists_build(t, l, theta, t->side, t->ev_level);
    if (rc) return rc;
    FMM_CUDA(cudaEventRecord(t->ev[0], t->side));
    const StepSync sync{t->side, t->ev[0], t->ev[1], t->ev[2]};
    return evaluate(t, l, q, *prm, phi, s, &sync);
}

int fmm_autotune(fmm_tree t, fmm_lists l, const double* q, const fmm_params* prm, double* phi, void* stream,
                 int* m2l_blocks, int* p2p_blocks)
{
    if (!t || !l || !q || !prm || !phi) return fail(FMM_ERR_ARG, "NULL argument");
    if (l->tree != t) return fail(FMM_ERR_STATE, "lists were created for another tree");
    if (!t->built || !l->built) return fail(FMM_ERR_STATE, "tree or lists not built");
    if (prm->p < 0 || prm->p > 40) return fail(FMM_ERR_ARG, "p = %d outside [0, 40]", prm->p);
    if (prm->mode != FMM_MODE_FP64 && prm->mode != FMM_MODE_MIXED && prm->mode != FMM_MODE_SPLIT)
        return fail(FMM_ERR_ARG, "unknown mode %d", prm->mode);
    GUARD(t->dev);
    return autotune(t, l, q, *prm, phi, (cudaStream_t)stream, m2l_blocks, p2p_blocks);
}

int fmm_set_m2l_kernel(fmm_tree t, int kind)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (kind < 0 || kind > 2) return fail(FMM_ERR_ARG, "unknown M2L kernel %d", kind);
    t->m2l_kind = kind;
    return FMM_OK;
}

int fmm_get_m2l_kernel(fmm_tree t)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    return t->m2l_kind;
}

int fmm_set_m2l_shape(fmm_tree t, int chunk, int stages)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (chunk < 0 || chunk > 256) return fail(FMM_ERR_ARG, "M2L chunk %d outside [0, 256]", chunk);
    if (stages < 0 || stages > 2) return fail(FMM_ERR_ARG, "M2L stages %d outside [0, 2]", stages);
    t->tune_m2l_chunk = chunk;
    t->tune_m2l_stages = stages;
    return FMM_OK;
}

int fmm_get_m2l_shape(fmm_tree t, int* chunk, int* stages)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (chunk) *chunk = t->tune_m2l_chunk;
    if (stages) *stages = t->tune_m2l_stages;
    return FMM_OK;
}

int fmm_set_near_shape(fmm_tree t, int targets)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (targets != 0 && targets != 2 && targets != 4)
        return fail(FMM_ERR_ARG, "near-field targets per lane %d: 0, 2 or 4", targets);
    t->tune_p2p_nt = targets;
    return FMM_OK;
}

int fmm_get_near_shape(fmm_tree t, int* targets)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (targets) *targets = t->tune_p2p_nt;
    return FMM_OK;
}

int fmm_set_launch(fmm_tree t, int m2l_blocks, int p2p_blocks)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    if (m2l_blocks < 0 || p2p_blocks < 0 || m2l_blocks > 65535 || p2p_blocks > 65535)
        return fail(FMM_ERR_ARG, "block counts must lie in [0, 65535]");
    GUARD(t->dev);
    t->tune_m2l_blocks = m2l_blocks;
    t->tune_p2p_blocks = p2p_blocks;
    return sched_tuned(t);
}

int fmm_evaluate_field(fmm_tree t, fmm_lists l, const double* q, const fmm_params* prm, double* fre,
                       double* fim, void* stream)
{
    if (!t || !l || !q || !prm || !fre || !fim) return fail(FMM_ERR_ARG, "NULL argument");
    if (l->tree != t) return fail(FMM_ERR_STATE, "lists were created for another tree");
    if (!t->built || !l->built) return fail(FMM_ERR_STATE, "tree or lists not built");
    if (prm->p < 0 || prm->p > 40) return fail(FMM_ERR_ARG, "p = %d outside [0, 40]", prm->p);
    if (prm->mode != FMM_MODE_FP64 && prm->mode != FMM_MODE_MIXED && prm->mode != FMM_MODE_SPLIT)
        return fail(FMM_ERR_ARG, "unknown mode %d", prm->mode);
    GUARD(t->dev);
    return evaluate_field(t, l, q, *prm, fre, fim, (cudaStream_t)stream);
}

int fmm_direct_field(const double* x, const double* y, const double* q, int64_t n, const int64_t* targets,
                     int64_t m, double* fre, double* fim, void* stream)
{
    if (!x || !y || !q || (m > 0 && (!targets || !fre || !fim))) return fail(FMM_ERR_ARG, "NULL argument");
    if (n < 1 || m < 0) return fail(FMM_ERR_ARG, "bad sizes n = %lld, m = %lld", (long long)n, (long long)m);
    return direct_field(x, y, q, n, targets, m, fre, fim, (cudaStream_t)stream);
}

int fmm_direct(const double* x, const double* y, const double* q, int64_t n, const int64_t* targets,
               int64_t m, double* phi, void* stream)
{
    if (!x || !y || !q || (m > 0 && (!targets || !phi))) return fail(FMM_ERR_ARG, "NULL argument");
    if (n < 1 || m < 0) return fail(FMM_ERR_ARG, "bad sizes n = %lld, m = %lld", (long long)n, (long long)m);
    return direct(x, y, q, n, targets, m, phi, (cudaStream_t)stream);
}

int fmm_sync_status(fmm_tree t, fmm_lists l, void* stream)
{
    if (!t) return fail(FMM_ERR_ARG, "NULL tree");
    GUARD(t->dev);
    FMM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int32_t st = 0, sl = 0;
    FMM_CUDA(cudaMemcpy(&st, t->status, 4, cudaMemcpyDeviceToHost));
    FMM_CUDA(cudaMemset(t->status, 0, 4));
    if (l) {
        FMM_CUDA(cudaMemcpy(&sl, l->status, 4, cudaMemcpyDeviceToHost));
        FMM_CUDA(cudaMemset(l->status, 0, 4));
    }
    return status_to_code(st | sl);
}

}  // extern "C"
