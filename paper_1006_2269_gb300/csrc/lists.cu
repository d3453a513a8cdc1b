// Interaction lists on the GPU: the connectivity rule of Section 4 with the theta-criterion
// (Criterion 2.1).  Level by level, one warp per box tests the children of its parent's strong
// list (one lane per candidate) and compacts the outcome with ballots, so every list comes out in
// ascending candidate order.  A count pass, a device-wide scan and a fill pass turn the counts
// into CSR offsets; the running total of each level is read from device memory, so the whole
// build is asynchronous.  Storage is preallocated: entries beyond the capacity are dropped and
// reported through the status word, and later levels never read past the capacity.
#include <algorithm>

#include "common.cuh"

namespace fmm {
namespace {

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

__global__ void k_lists_root(int32_t* woff, int32_t* soff, int32_t* sidx)
{
    if (threadIdx.x == 0) {
        woff[0] = 0;
        woff[1] = 0;
        soff[0] = 0;
        soff[1] = 1;
        sidx[0] = 0;
    }
}

template <bool FILL>
__global__ void __launch_bounds__(256) k_lists(int l, const double* __restrict__ cen,
                                               const double* __restrict__ rad, double theta,
                                               const int32_t* __restrict__ woff, int32_t* __restrict__ widx,
                                               int64_t wcap, const int32_t* __restrict__ soff,
                                               int32_t* __restrict__ sidx, int64_t scap,
                                               int32_t* __restrict__ wcnt, int32_t* __restrict__ scnt)
{
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= level_size(l)) return;
    const int64_t base = level_base(l), g = base + b;
    const int64_t pg = level_base(l - 1) + (b >> 2);
    const int64_t s0 = min((int64_t)soff[pg], scap), s1 = min((int64_t)soff[pg + 1], scap);
    const int64_t ncand = s1 > s0 ? 4 * (s1 - s0) : 0;
    const double cx = cen[2 * g], cy = cen[2 * g + 1], r = rad[g];
    const unsigned lt = lanemask_lt();
    int64_t wpos = FILL ? woff[g] : 0, spos = FILL ? soff[g] : 0;
    int nw = 0, ns = 0;
    for (int64_t c0 = 0; c0 < ncand; c0 += 32) {
        int64_t c = c0 + lane;
        bool valid = c < ncand;
        int32_t cand = 0;
        bool weak = false;
        if (valid) {
            cand = 4 * sidx[s0 + (c >> 2)] + (int32_t)(c & 3);
            int64_t cg = base + cand;
            weak = theta_weak(cx, cy, r, cen[2 * cg], cen[2 * cg + 1], rad[cg], theta);
        }
        unsigned bw = __ballot_sync(0xffffffffu, valid && weak);
        unsigned bs = __ballot_sync(0xffffffffu, valid && !weak);
        if (FILL && valid) {
            if (weak) {
                int64_t p = wpos + nw + __popc(bw & lt);
                if (p < wcap) widx[p] = cand;
            } else {
                int64_t p = spos + ns + __popc(bs & lt);
                if (p < scap) sidx[p] = cand;
            }
        }
        nw += __popc(bw);
        ns += __popc(bs);
    }
    if (!FILL && lane == 0) {
        wcnt[b] = nw;
        scnt[b] = ns;
    }
}

__global__ void k_lists_check(const int32_t* woff, const int32_t* soff, int64_t nbox, int64_t wcap,
                              int64_t scap, int32_t* status)
{
    if (threadIdx.x == 0 && ((int64_t)woff[nbox] > wcap || (int64_t)soff[nbox] > scap ||
                             woff[nbox] == INT32_MAX || soff[nbox] == INT32_MAX))
        atomicOr(status, ST_CAPACITY);
}

}  // namespace

int lists_build(fmm_tree t, fmm_lists li, double theta, cudaStream_t s)
{
    const int L = t->L;
    StageScope scope(FMM_STAGE_LISTS, s);
    k_lists_root<<<1, 32, 0, s>>>(li->woff, li->soff, li->sidx); note_launch();
    for (int l = 1; l <= L; l++) {
        int64_t nb = level_size(l);
        unsigned blocks = (unsigned)((nb * 32 + 255) / 256);
        k_lists<false><<<blocks, 256, 0, s>>>(l, t->centers, t->radii, theta, li->woff, li->widx,
                                              li->wcap, li->soff, li->sidx, li->scap, li->wcnt,
                                              li->scnt); note_launch();
        int64_t base = level_base(l);
        int rc = scan_with_base(li->wcnt, nb, li->woff + base, li->woff + base, li->scan_tmp, s);
        if (rc) return rc;
        rc = scan_with_base(li->scnt, nb, li->soff + base, li->soff + base, li->scan_tmp, s);
        if (rc) return rc;
        k_lists<true><<<blocks, 256, 0, s>>>(l, t->centers, t->radii, theta, li->woff, li->widx,
                                             li->wcap, li->soff, li->sidx, li->scap, li->wcnt,
                                             li->scnt); note_launch();
        FMM_LAUNCH_CHECK("lists");
    }
    k_lists_check<<<1, 32, 0, s>>>(li->woff, li->soff, t->nbox, li->wcap, li->scap, li->status); note_launch();
    FMM_LAUNCH_CHECK("lists: check");
    li->theta = theta;
    li->built = true;
    return 0;
}

}  // namespace fmm
