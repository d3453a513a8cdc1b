// Expansions and evaluation (Section 4; classical complex representation of Section 5).
//
// Storage is radius-scaled: a box of centre c and radius rho keeps a~_k = a_k / rho^k (multipole)
// and b~_l = b_l * rho^l (local), and points enter through xi = (z - c) / rho (taken as 0 when
// rho = 0).  In scaled form every shift is a combination of quantities of modulus <= 1:
//   P2M  a~_0 = sum q_j,  a~_k = -sum q_j xi_j^k / k
//   M2M  b~_l = -a_0 w^l / l + sum_{k=1..l} a~_k C(l-1,k-1) s^k w^(l-k),
//        w = (c_child - c_parent)/rho_p, s = rho_c/rho_p
//   M2L  with z0 = c_src - c_tgt, u = -rho_s/z0, v = rho_t/z0 (|u| + |v| <= theta):
//        b~_0 = a_0 log|z0| + sum_k a~_k u^k,
//        b~_l = v^l [ -a_0/l + sum_k C(l+k-1,k-1) a~_k u^k ]
//        evaluated as (2v)^l * sum_k M'[l][k] * (a~_k (2u)^k) with the fixed matrix
//        M'[l][k] = C(l+k-1,k-1) / 2^(l+k) (k >= 1), M'[l][0] = -1/(l 2^l), whose entries are <= 1/2
//        (the "diagonal scaling x constant Pascal matrix x diagonal scaling" form of Section 4)
//   L2L  b~'_l = s^l sum_{k>=l} b~_k C(k,l) w^(k-l)
//   L2P  phi += Re sum_l b~_l xi^l
// Only the real part of the potential is needed, so the imaginary part of log(-z0) is dropped.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace fmm {

constexpr int PMAXC = 41;  // p <= 40

__constant__ double c_md[PMAXC][PMAXC];     // M'[l][k] in binary64
__constant__ float c_mf[PMAXC][PMAXC];      // M'[l][k] rounded to binary32
__constant__ double c_binom[PMAXC][PMAXC];  // C(n, k), n < PMAXC

namespace {

template <typename T>
struct alignas(2 * sizeof(T)) cx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.re * s, a.im * s}; }
// a*b + c
template <typename T>
__device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> c)
{
    return {c.re + a.re * b.re - a.im * b.im, c.im + a.re * b.im + a.im * b.re};
}

template <typename T>
__device__ __forceinline__ T mtab(int l, int k);
template <>
__device__ __forceinline__ double mtab<double>(int l, int k) { return c_md[l][k]; }
template <>
__device__ __forceinline__ float mtab<float>(int l, int k) { return c_mf[l][k]; }

template <typename T>
__device__ __forceinline__ T ipow(T x, int e)
{
    T r = 1;
    while (e) {
        if (e & 1) r *= x;
        x *= x;
        e >>= 1;
    }
    return r;
}

__device__ __forceinline__ int level_of(int64_t g)
{
    int l = 0;
    while (level_base(l + 1) <= g) l++;
    return l;
}

// z0 = c_src - c_tgt: in binary64 directly, in binary32 from the float-float centres so that
// the difference of two nearby centres keeps its relative accuracy.
template <typename T>
struct Geo;
template <>
struct Geo<double> {
    const double* cen;
    __device__ __forceinline__ cx<double> diff(int64_t a, int64_t b) const
    {
        return {cen[2 * a] - cen[2 * b], cen[2 * a + 1] - cen[2 * b + 1]};
    }
};
template <>
struct Geo<float> {
    const float* hi;
    const float* lo;
    __device__ __forceinline__ cx<float> diff(int64_t a, int64_t b) const
    {
        float2 ha = *(const float2*)(hi + 2 * a), hb = *(const float2*)(hi + 2 * b);
        float2 la = *(const float2*)(lo + 2 * a), lb = *(const float2*)(lo + 2 * b);
        return {(ha.x - hb.x) + (la.x - lb.x), (ha.y - hb.y) + (la.y - lb.y)};
    }
};

__device__ __forceinline__ double log_d(double x) { return log(x); }
__device__ __forceinline__ float log_d(float x) { return logf(x); }

// ---- strengths in canonical order ----
template <typename T>
__global__ void k_gather_q(const int32_t* __restrict__ perm, const double* __restrict__ q, int64_t n,
                           T* __restrict__ qs, int32_t* status)
{
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = q[perm[i]];
        bad |= !isfinite(v);
        qs[i] = (T)v;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// ---- P2M: one warp per leaf, one lane per point; column sums through shared memory ----
template <typename T>
__global__ void k_p2m(int L, int P, int PS, const int32_t* __restrict__ lb, const T* __restrict__ qs,
                      const double* __restrict__ xs, const double* __restrict__ ys,
                      const float* __restrict__ dxf, const float* __restrict__ dyf,
                      const double* __restrict__ cen, const double* __restrict__ rad,
                      cx<T>* __restrict__ Me)
{
    extern __shared__ unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * wpb + w;
    if (b >= level_size(L)) return;
    cx<T>* S = (cx<T>*)smem + (size_t)w * 33 * P;
    const int64_t g = level_base(L) + b;
    const double rho = rad[g];
    const int32_t t0 = lb[b], t1 = lb[b + 1];
    cx<T> acc[2] = {{0, 0}, {0, 0}};
    for (int32_t tb = t0; tb < t1; tb += 32) {
        const int32_t t = tb + lane;
        T xr = 0, xi = 0, qq = 0;
        if (t < t1) {
            qq = qs[t];
            if (rho > 0) {
                if (sizeof(T) == 8) {
                    xr = (T)((xs[t] - cen[2 * g]) / rho);
                    xi = (T)((ys[t] - cen[2 * g + 1]) / rho);
                } else {
                    const T inv = (T)(1.0 / rho);
                    xr = (T)dxf[t] * inv;
                    xi = (T)dyf[t] * inv;
                }
            }
        }
        cx<T> pw = {qq, 0};
        const cx<T> xi_c = {xr, xi};
        for (int k = 0; k < P; k++) {
            S[k * 33 + lane] = pw;
            pw = cmul(pw, xi_c);
        }
        __syncwarp();
        for (int k = lane, s = 0; k < P; k += 32, s++) {
            cx<T> sum = {0, 0};
            for (int j = 0; j < 32; j++) sum = cadd(sum, S[k * 33 + j]);
            acc[s] = cadd(acc[s], sum);
        }
        __syncwarp();
    }
    for (int k = lane, s = 0; k < P; k += 32, s++)
        Me[g * PS + k] = k == 0 ? acc[s] : cscale(acc[s], (T)(-1.0 / k));
}

// ---- M2M: one warp per parent, one lane per output coefficient ----
template <typename T>
__global__ void k_m2m(int l, int P, int PS, const double* __restrict__ cen,
                      const double* __restrict__ rad, cx<T>* __restrict__ Me)
{
    extern __shared__ unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * wpb + w;
    if (b >= level_size(l)) return;
    cx<T>* D = (cx<T>*)smem + (size_t)w * P;
    const int64_t g = level_base(l) + b;
    const double rp = rad[g];
    cx<T> acc[2] = {{0, 0}, {0, 0}};
    for (int k = 0; k < 4; k++) {
        const int64_t cg = level_base(l + 1) + 4 * b + k;
        cx<T> wv = {0, 0};
        T s = 0;
        if (rp > 0) {
            wv = {(T)((cen[2 * cg] - cen[2 * g]) / rp), (T)((cen[2 * cg + 1] - cen[2 * g + 1]) / rp)};
            s = (T)(rad[cg] / rp);
        }
        for (int j = lane; j < P; j += 32) D[j] = cscale(Me[cg * PS + j], ipow(s, j));
        __syncwarp();
        for (int o = lane, si = 0; o < P; o += 32, si++) {
            cx<T> h;
            if (o == 0) {
                h = D[0];
            } else {
                h = cscale(D[0], (T)(-1.0 / o));
                for (int j = 1; j <= o; j++) h = cfma(h, wv, cscale(D[j], (T)c_binom[o - 1][j - 1]));
            }
            acc[si] = cadd(acc[si], h);
        }
        __syncwarp();
    }
    for (int o = lane, si = 0; o < P; o += 32, si++) Me[g * PS + o] = acc[si];
}

// ---- M2L, one thread per target box of levels 1..L (runtime P; operands in shared memory) ----
template <typename T>
__global__ void k_m2l_generic(int64_t g0, int64_t g1, int P, int PS, const int32_t* __restrict__ woff,
                              const int32_t* __restrict__ widx, int64_t wcap, Geo<T> geo,
                              const double* __restrict__ rad, const cx<T>* __restrict__ Me,
                              cx<T>* __restrict__ Le)
{
    extern __shared__ unsigned char smem[];
    const int nt = blockDim.x, tid = threadIdx.x;
    cx<T>* X = (cx<T>*)smem;            // X[k * nt + tid]
    cx<T>* A = X + (size_t)P * nt;      // A[l * nt + tid]
    const int64_t g = g0 + (int64_t)blockIdx.x * nt + tid;
    if (g >= g1) return;
    const int l = level_of(g);
    const int64_t base = level_base(l);
    for (int j = 0; j < P; j++) A[j * nt + tid] = {0, 0};
    const T rt = (T)rad[g];
    const int64_t e0 = min((int64_t)woff[g], wcap), e1 = min((int64_t)woff[g + 1], wcap);
    for (int64_t e = e0; e < e1; e++) {
        const int64_t sg = base + widx[e];
        const cx<T> z0 = geo.diff(sg, g);
        const T r2 = z0.re * z0.re + z0.im * z0.im;
        const T ir2 = (T)1 / r2;
        const cx<T> inv = {z0.re * ir2, -z0.im * ir2};
        const T rs = (T)rad[sg];
        const cx<T> u2 = cscale(inv, (T)(-2) * rs), v2 = cscale(inv, (T)2 * rt);
        const T a0 = Me[sg * PS].re;
        X[tid] = {a0, 0};
        cx<T> up = u2;
        for (int k = 1; k < P; k++) {
            X[k * nt + tid] = cmul(Me[sg * PS + k], up);
            up = cmul(up, u2);
        }
        cx<T> vp = {1, 0};
        for (int o = 0; o < P; o++) {
            cx<T> y = {0, 0};
            for (int k = 0; k < P; k++) {
                const T m = mtab<T>(o, k);
                const cx<T> x = X[k * nt + tid];
                y.re += m * x.re;
                y.im += m * x.im;
            }
            if (o == 0) y.re += a0 * (T)0.5 * log_d(r2);
            A[o * nt + tid] = cfma(vp, y, A[o * nt + tid]);
            vp = cmul(vp, v2);
        }
    }
    for (int o = 0; o < P; o++) Le[g * PS + o] = A[o * nt + tid];
}

// ---- M2L, binary32, compile-time P: the scaled source coefficients and the accumulators live
// in registers and the constant matrix is read from the constant bank by the unrolled loop ----
template <int P>
__global__ void __launch_bounds__(128) k_m2l_f32(int64_t g0, int64_t g1, int PS,
                                                 const int32_t* __restrict__ woff,
                                                 const int32_t* __restrict__ widx, int64_t wcap,
                                                 Geo<float> geo, const double* __restrict__ rad,
                                                 const cx<float>* __restrict__ Me,
                                                 cx<float>* __restrict__ Le)
{
    const int64_t g = g0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= g1) return;
    const int l = level_of(g);
    const int64_t base = level_base(l);
    cx<float> acc[P];
#pragma unroll
    for (int j = 0; j < P; j++) acc[j] = {0.f, 0.f};
    const float rt = (float)rad[g];
    const int64_t e0 = min((int64_t)woff[g], wcap), e1 = min((int64_t)woff[g + 1], wcap);
    for (int64_t e = e0; e < e1; e++) {
        const int64_t sg = base + widx[e];
        const cx<float> z0 = geo.diff(sg, g);
        const float r2 = z0.re * z0.re + z0.im * z0.im;
        const float ir2 = 1.f / r2;
        const cx<float> inv = {z0.re * ir2, -z0.im * ir2};
        const float rs = (float)rad[sg];
        const cx<float> u2 = cscale(inv, -2.f * rs), v2 = cscale(inv, 2.f * rt);
        const cx<float>* src = Me + sg * PS;
        cx<float> x[P];
        x[0] = {src[0].re, 0.f};
        cx<float> up = u2;
#pragma unroll
        for (int k = 1; k < P; k++) {
            x[k] = cmul(src[k], up);
            up = cmul(up, u2);
        }
        cx<float> vp = {1.f, 0.f};
#pragma unroll
        for (int o = 0; o < P; o++) {
            cx<float> y = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < P; k++) {
                y.re = fmaf(c_mf[o][k], x[k].re, y.re);
                y.im = fmaf(c_mf[o][k], x[k].im, y.im);
            }
            if (o == 0) y.re = fmaf(x[0].re * 0.5f, logf(r2), y.re);
            acc[o] = cfma(vp, y, acc[o]);
            vp = cmul(vp, v2);
        }
    }
#pragma unroll
    for (int o = 0; o < P; o++) Le[g * PS + o] = acc[o];
}

// ---- L2L: one warp per child box of level l+1 ----
template <typename T>
__global__ void k_l2l(int l, int P, int PS, const double* __restrict__ cen, const double* __restrict__ rad,
                      cx<T>* __restrict__ Le)
{
    extern __shared__ unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * wpb + w;
    if (c >= level_size(l + 1)) return;
    cx<T>* B = (cx<T>*)smem + (size_t)w * P;
    const int64_t cg = level_base(l + 1) + c, pg = level_base(l) + (c >> 2);
    const double rp = rad[pg];
    cx<T> wv = {0, 0};
    T s = 0;
    if (rp > 0) {
        wv = {(T)((cen[2 * cg] - cen[2 * pg]) / rp), (T)((cen[2 * cg + 1] - cen[2 * pg + 1]) / rp)};
        s = (T)(rad[cg] / rp);
    }
    for (int j = lane; j < P; j += 32) B[j] = Le[pg * PS + j];
    __syncwarp();
    for (int o = lane; o < P; o += 32) {
        cx<T> h = cscale(B[P - 1], (T)c_binom[P - 1][o]);
        for (int k = P - 2; k >= o; k--) h = cfma(h, wv, cscale(B[k], (T)c_binom[k][o]));
        const cx<T> r = cscale(h, ipow(s, o));
        Le[cg * PS + o] = cadd(Le[cg * PS + o], r);
    }
}

// ---- L2P + near field: one warp per leaf, one lane per target; source tiles of 32 points are
// staged in shared memory and read by every lane.  Potentials are written in input order. ----
template <typename T>
__global__ void k_leaf_eval(int L, int P, int PS, const int32_t* __restrict__ lb,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ soff,
                            const int32_t* __restrict__ sidx, int64_t scap, const double* __restrict__ xs,
                            const double* __restrict__ ys, const float* __restrict__ dxf,
                            const float* __restrict__ dyf, const T* __restrict__ qs,
                            const double* __restrict__ cen, const float* __restrict__ chi,
                            const float* __restrict__ clo, const double* __restrict__ rad,
                            const cx<T>* __restrict__ Le, double* __restrict__ phi)
{
    extern __shared__ unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * wpb + w;
    if (b >= level_size(L)) return;
    cx<T>* B = (cx<T>*)smem + (size_t)w * (P + 48);
    T* sx = (T*)(B + P);
    T* sy = sx + 32;
    T* sq = sy + 32;
    const int64_t g = level_base(L) + b;
    for (int j = lane; j < P; j += 32) B[j] = Le[g * PS + j];
    const double rho = rad[g];
    const int32_t t0 = lb[b], t1 = lb[b + 1];
    const int64_t e0 = min((int64_t)soff[g], scap), e1 = min((int64_t)soff[g + 1], scap);
    const bool f32 = sizeof(T) == 4;
    __syncwarp();
    for (int32_t tb = t0; tb < t1; tb += 32) {
        const int32_t t = tb + lane;
        const bool valid = t < t1;
        T xi = 0, yi = 0;  // target: absolute (binary64) or offset from the leaf centre (binary32)
        T far = 0;
        if (valid) {
            xi = f32 ? (T)dxf[t] : (T)xs[t];
            yi = f32 ? (T)dyf[t] : (T)ys[t];
            cx<T> z = {0, 0};
            if (rho > 0) {
                if (f32) {
                    const T inv = (T)(1.0 / rho);
                    z = {xi * inv, yi * inv};
                } else {
                    z = {(T)((xs[t] - cen[2 * g]) / rho), (T)((ys[t] - cen[2 * g + 1]) / rho)};
                }
            }
            cx<T> h = B[P - 1];
            for (int k = P - 2; k >= 0; k--) h = cfma(h, z, B[k]);
            far = h.re;
        }
        T near = 0;
        for (int64_t e = e0; e < e1; e++) {
            const int64_t sb = sidx[e];
            T ox = 0, oy = 0;  // binary32: centre of the source leaf relative to the target leaf
            if (f32) {
                const int64_t sg = level_base(L) + sb;
                ox = (T)((chi[2 * sg] - chi[2 * g]) + (clo[2 * sg] - clo[2 * g]));
                oy = (T)((chi[2 * sg + 1] - chi[2 * g + 1]) + (clo[2 * sg + 1] - clo[2 * g + 1]));
            }
            const int32_t s0 = lb[sb], s1 = lb[sb + 1];
            for (int32_t sc = s0; sc < s1; sc += 32) {
                const int32_t s = sc + lane;
                if (s < s1) {
                    sx[lane] = f32 ? (T)dxf[s] + ox : (T)xs[s];
                    sy[lane] = f32 ? (T)dyf[s] + oy : (T)ys[s];
                    sq[lane] = qs[s];
                }
                __syncwarp();
                const int cnt = min(32, s1 - sc);
                for (int j = 0; j < cnt; j++) {
                    const T dx = xi - sx[j], dy = yi - sy[j];
                    const T r2 = dx * dx + dy * dy;
                    if (r2 > (T)0) near += sq[j] * (f32 ? (T)__log2f((float)r2) : (T)log((double)r2));
                }
                __syncwarp();
            }
        }
        if (valid) {
            const T scale = f32 ? (T)(0.5 * 0.69314718055994530942) : (T)0.5;
            phi[perm[t]] = (double)far + (double)(near * scale);
        }
    }
}

// ---- direct sum at sampled targets (binary64), one block per target ----
__global__ void k_direct(const double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ q, int64_t n, const int64_t* __restrict__ tgt,
                         double* __restrict__ phi)
{
    __shared__ double red[32];
    const int64_t i = tgt[blockIdx.x];
    const double xi = x[i], yi = y[i];
    double s = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double dx = xi - x[j], dy = yi - y[j];
        if (j != i && (dx != 0.0 || dy != 0.0)) s += q[j] * log(hypot(dx, dy));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) phi[blockIdx.x] = s;
    }
}

// ---- per-device constant tables ----
std::mutex g_tab_mutex;
bool g_tab_ready[128] = {};

int ensure_tables()
{
    int dev = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_tab_mutex);
    if (dev < 0 || dev >= 128) return fail(FMM_ERR_ARG, "device ordinal %d out of range", dev);
    if (g_tab_ready[dev]) return 0;
    static double bn[PMAXC][PMAXC], md[PMAXC][PMAXC];
    static float mf[PMAXC][PMAXC];
    // binomials by Pascal's rule (exact while below 2^53)
    static double big[2 * PMAXC + 2][2 * PMAXC + 2];
    for (int i = 0; i < 2 * PMAXC + 2; i++)
        for (int j = 0; j < 2 * PMAXC + 2; j++)
            big[i][j] = j == 0 ? 1.0 : (i == 0 ? 0.0 : big[i - 1][j - 1] + big[i - 1][j]);
    for (int i = 0; i < PMAXC; i++)
        for (int j = 0; j < PMAXC; j++) bn[i][j] = big[i][j];
    for (int l = 0; l < PMAXC; l++)
        for (int k = 0; k < PMAXC; k++) {
            double v;
            if (k == 0)
                v = l == 0 ? 0.0 : -1.0 / ((double)l * ldexp(1.0, l));
            else
                v = ldexp(big[l + k - 1][k - 1], -(l + k));
            md[l][k] = v;
            mf[l][k] = (float)v;
        }
    FMM_CUDA(cudaMemcpyToSymbol(c_binom, bn, sizeof(bn)));
    FMM_CUDA(cudaMemcpyToSymbol(c_md, md, sizeof(md)));
    FMM_CUDA(cudaMemcpyToSymbol(c_mf, mf, sizeof(mf)));
    g_tab_ready[dev] = true;
    return 0;
}

int alloc_ws(fmm_tree t, int PS, bool f64)
{
    int& have = f64 ? t->ws_ps64 : t->ws_ps32;
    if (have >= PS) return 0;
    void** M = f64 ? &t->Me : &t->Mf;
    void** Lc = f64 ? &t->Le : &t->Lf;
    const size_t csz = f64 ? 16 : 8;
    cudaFree(*M);
    cudaFree(*Lc);
    *M = *Lc = nullptr;
    have = 0;
    const size_t bytes = (size_t)t->nbox * PS * csz;
    if (cudaMalloc(M, bytes) != cudaSuccess || cudaMalloc(Lc, bytes) != cudaSuccess)
        return fail(FMM_ERR_OOM, "expansion workspace of %zu bytes", 2 * bytes);
    if (f64 && !t->qs && cudaMalloc((void**)&t->qs, 8 * (size_t)t->n) != cudaSuccess)
        return fail(FMM_ERR_OOM, "strength workspace");
    if (!f64 && !t->qf && cudaMalloc((void**)&t->qf, 4 * (size_t)t->n) != cudaSuccess)
        return fail(FMM_ERR_OOM, "strength workspace");
    have = PS;
    return 0;
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

template <typename T>
int run(fmm_tree t, fmm_lists li, const double* q, int P, double* phi, cudaStream_t s)
{
    const bool f64 = sizeof(T) == 8;
    const int PS = (P + 1) & ~1;
    int rc = alloc_ws(t, PS, f64);
    if (rc) return rc;
    cx<T>* Me = (cx<T>*)(f64 ? t->Me : t->Mf);
    cx<T>* Le = (cx<T>*)(f64 ? t->Le : t->Lf);
    T* qs = f64 ? (T*)t->qs : (T*)t->qf;
    const int L = t->L;
    const int64_t n = t->n;

    {
        StageScope scope(FMM_STAGE_GATHER, s);
        k_gather_q<T><<<grid_for(n, 256), 256, 0, s>>>(t->perm, q, n, qs, t->status); note_launch();
        FMM_LAUNCH_CHECK("evaluate: gather");
    }

    const int WPB = 4;
    if (L >= 1) {
        // upward pass
        const int64_t nleaf = level_size(L);
        size_t sm = (size_t)WPB * 33 * P * sizeof(cx<T>);
        FMM_CUDA(cudaFuncSetAttribute(k_p2m<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        {
            StageScope scope(FMM_STAGE_P2M, s);
            k_p2m<T><<<(unsigned)((nleaf + WPB - 1) / WPB), 32 * WPB, sm, s>>>(
                L, P, PS, t->leaf_begin, qs, t->xs, t->ys, t->dxf, t->dyf, t->centers, t->radii, Me); note_launch();
        }
        StageScope m2m_scope(FMM_STAGE_M2M, s);
        for (int l = L - 1; l >= 1; l--) {
            const int64_t nb = level_size(l);
            k_m2m<T><<<(unsigned)((nb + WPB - 1) / WPB), 32 * WPB, WPB * P * sizeof(cx<T>), s>>>(
                l, P, PS, t->centers, t->radii, Me); note_launch();
        }
        FMM_LAUNCH_CHECK("evaluate: upward pass");
        prof_mark(FMM_STAGE_M2M, false, s);
        m2m_scope.stage = -1;

        // M2L on the weak lists of every level (one launch over levels 1..L)
        const int64_t g0 = 1, g1 = t->nbox;
        bool done = false;
        prof_mark(FMM_STAGE_M2L, true, s);
        if (!f64) {
            Geo<float> geo{t->cen_hi, t->cen_lo};
            const unsigned blocks = (unsigned)((g1 - g0 + 127) / 128);
            const cx<float>* Mf = (const cx<float>*)Me;
            cx<float>* Lf = (cx<float>*)Le;
            done = true;
            switch (P) {
                case 17: k_m2l_f32<17><<<blocks, 128, 0, s>>>(g0, g1, PS, li->woff, li->widx, li->wcap, geo, t->radii, Mf, Lf); note_launch(); break;
                case 18: k_m2l_f32<18><<<blocks, 128, 0, s>>>(g0, g1, PS, li->woff, li->widx, li->wcap, geo, t->radii, Mf, Lf); note_launch(); break;
                case 21: k_m2l_f32<21><<<blocks, 128, 0, s>>>(g0, g1, PS, li->woff, li->widx, li->wcap, geo, t->radii, Mf, Lf); note_launch(); break;
                case 31: k_m2l_f32<31><<<blocks, 128, 0, s>>>(g0, g1, PS, li->woff, li->widx, li->wcap, geo, t->radii, Mf, Lf); note_launch(); break;
                default: done = false;
            }
        }
        if (!done) {
            const int NT = 64;
            size_t sm2 = (size_t)2 * P * NT * sizeof(cx<T>);
            FMM_CUDA(cudaFuncSetAttribute(k_m2l_generic<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
            Geo<T> geo;
            if constexpr (sizeof(T) == 8) geo = Geo<T>{t->centers};
            else geo = Geo<T>{t->cen_hi, t->cen_lo};
            k_m2l_generic<T><<<(unsigned)((g1 - g0 + NT - 1) / NT), NT, sm2, s>>>(
                g0, g1, P, PS, li->woff, li->widx, li->wcap, geo, t->radii, Me, Le); note_launch();
        }
        prof_mark(FMM_STAGE_M2L, false, s);
        FMM_LAUNCH_CHECK("evaluate: M2L");

        // downward pass
        StageScope l2l_scope(FMM_STAGE_L2L, s);
        for (int l = 1; l < L; l++) {
            const int64_t nc = level_size(l + 1);
            k_l2l<T><<<(unsigned)((nc + WPB - 1) / WPB), 32 * WPB, WPB * P * sizeof(cx<T>), s>>>(
                l, P, PS, t->centers, t->radii, Le); note_launch();
        }
        FMM_LAUNCH_CHECK("evaluate: L2L");
    } else {
        FMM_CUDA(cudaMemsetAsync(Le, 0, PS * sizeof(cx<T>), s));
    }

    // L2P + near field on the leaves
    {
        StageScope scope(FMM_STAGE_LEAF, s);
        const int64_t nleaf = level_size(L);
        size_t sm = (size_t)WPB * ((P + 48) * sizeof(cx<T>));
        k_leaf_eval<T><<<(unsigned)((nleaf + WPB - 1) / WPB), 32 * WPB, sm, s>>>(
            L, P, PS, t->leaf_begin, t->perm, li->soff, li->sidx, li->scap, t->xs, t->ys, t->dxf,
            t->dyf, qs, t->centers, t->cen_hi, t->cen_lo, t->radii, Le, phi); note_launch();
        FMM_LAUNCH_CHECK("evaluate: leaf evaluation");
    }
    return 0;
}

}  // namespace

int evaluate(fmm_tree t, fmm_lists li, const double* q, const fmm_params& prm, double* phi,
             cudaStream_t s)
{
    int rc = ensure_tables();
    if (rc) return rc;
    const int P = prm.p + 1;
    if (prm.mode == FMM_MODE_FP64) return run<double>(t, li, q, P, phi, s);
    return run<float>(t, li, q, P, phi, s);
}

int direct(const double* x, const double* y, const double* q, int64_t n, const int64_t* tgt,
           int64_t m, double* phi, cudaStream_t s)
{
    if (m <= 0) return 0;
    for (int64_t off = 0; off < m; off += 65535) {
        const int64_t c = std::min<int64_t>(65535, m - off);
        k_direct<<<(unsigned)c, 256, 0, s>>>(x, y, q, n, tgt + off, phi + off); note_launch();
    }
    FMM_LAUNCH_CHECK("direct");
    return 0;
}

}  // namespace fmm
