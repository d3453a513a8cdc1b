// Input features of the parameter selector, computed from a built tree on the GPU.
//
// The balanced tree puts the same number of points in every box of a level (Section 4), so the
// distribution shows in the boxes' shapes instead: where points are dense the boxes are small,
// and elongated boxes (large aspect ratio) have long strong lists.  For every level l = 1..15 of
// an instance the features are four statistics over its 4^l boxes (long side s = max(w, h), short
// side max(min(w, h), 2^-30 s)):
//   [4(l-1) + 0]  mean of log2(s / s_root)          size scale
//   [4(l-1) + 1]  standard deviation of log2(s)     spread of sizes: non-uniformity
//   [4(l-1) + 2]  mean of log2(s / short side)      mean elongation
//   [4(l-1) + 3]  max of log2(s / short side)       worst elongation
// (zeros for levels the tree does not have), then [60] log10 N, [61] log10 tol, [62] levels / 16,
// [63] 0.  One block per (level, instance); binary64 sums.
#include "common.cuh"

namespace fmm {
namespace {

constexpr int FT = 256;

__device__ __forceinline__ void box_stats(const double* r, double root_long, double& lsz, double& lasp)
{
    const double w = r[1] - r[0], h = r[3] - r[2];
    const double s = fmax(fmax(w, h), 1e-300);
    const double sh = fmax(fmin(w, h), s * 0x1p-30);
    lsz = log2(s / root_long);
    lasp = log2(s / sh);
}

__global__ void __launch_bounds__(FT) k_features(const Inst* __restrict__ I, const double* __restrict__ rects,
                                                 double tol, float* __restrict__ out)
{
    const int l = blockIdx.x + 1, i = blockIdx.y;
    const Inst S = I[i];
    float* f = out + (int64_t)i * FMM_MLP_IN;
    if (l == 1 && threadIdx.x == 0) {
        f[FMM_FEAT_LOG10N] = (float)log10((double)S.n);
        f[FMM_FEAT_LOG10TOL] = (float)log10(tol);
        f[62] = (float)S.L / 16.f;
        f[63] = 0.f;
    }
    float* fl = f + 4 * (l - 1);
    if (l > S.L) {
        if (threadIdx.x < 4) fl[threadIdx.x] = 0.f;
        return;
    }
    const double* R = rects + 4 * S.b0;
    const double root_long = fmax(fmax(R[1] - R[0], R[3] - R[2]), 1e-300);
    double s1 = 0, s2 = 0, a1 = 0, amax = 0, sz1 = 0;
    const int64_t nb = level_size(l), base = level_base(l);
    for (int64_t b = threadIdx.x; b < nb; b += FT) {
        double lsz, lasp;
        box_stats(R + 4 * (base + b), root_long, lsz, lasp);
        sz1 += lsz;
        s1 += lsz;
        s2 += lsz * lsz;
        a1 += lasp;
        amax = fmax(amax, lasp);
    }
    __shared__ double red[4][FT];
    red[0][threadIdx.x] = s1;
    red[1][threadIdx.x] = s2;
    red[2][threadIdx.x] = a1;
    red[3][threadIdx.x] = amax;
    __syncthreads();
    for (int o = FT / 2; o; o >>= 1) {
        if (threadIdx.x < o) {
            red[0][threadIdx.x] += red[0][threadIdx.x + o];
            red[1][threadIdx.x] += red[1][threadIdx.x + o];
            red[2][threadIdx.x] += red[2][threadIdx.x + o];
            red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = red[0][0] / (double)nb;
        const double var = fmax(red[1][0] / (double)nb - m * m, 0.0);
        fl[0] = (float)m;
        fl[1] = (float)sqrt(var);
        fl[2] = (float)(red[2][0] / (double)nb);
        fl[3] = (float)red[3][0];
    }
    (void)sz1;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" int fmm_selector_features(fmm_tree t, double tol, float* features, void* stream)
{
    if (!t || !features) return fail(FMM_ERR_ARG, "NULL argument");
    if (!t->built) return fail(FMM_ERR_STATE, "tree not built");
    if (!(tol > 0.0 && tol < 1.0)) return fail(FMM_ERR_ARG, "tol = %g outside (0, 1)", tol);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != t->dev)
        return fail(FMM_ERR_STATE, "the tree's device must be current");
    k_features<<<dim3(15, t->n_inst), FT, 0, (cudaStream_t)stream>>>(t->dinst, t->rects, tol, features);
    note_launch();
    FMM_LAUNCH_CHECK("selector features");
    return FMM_OK;
}
