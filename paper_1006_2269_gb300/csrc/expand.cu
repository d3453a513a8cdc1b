// Expansions and evaluation (Section 4; classical complex representation of Section 5).
//
// Storage is radius-scaled: a box of centre c and radius rho keeps a~_k = a_k / rho^k (multipole)
// and b~_l = b_l * rho^l (local), and points enter through xi = (z - c) / rho (taken as 0 when
// rho = 0).  In scaled form every shift combines quantities of modulus <= 1:
//   P2M  a~_0 = sum q_j,  a~_k = -sum q_j xi_j^k / k
//   M2M  b~_l = -a_0 w^l / l + sum_{k=1..l} a~_k C(l-1,k-1) s^k w^(l-k),
//        w = (c_child - c_parent)/rho_p, s = rho_c/rho_p
//   M2L  with z0 = c_src - c_tgt, u = -rho_s/z0, v = rho_t/z0 (|u| + |v| <= theta < 1):
//        b~_0 = a_0 log|z0| + sum_k a~_k u^k,
//        b~_l = v^l [ -a_0/l + sum_k C(l+k-1,k-1) a~_k u^k ]
//        evaluated as (2v)^l * sum_k M'[l][k] * (a~_k (2u)^k) with the fixed matrix
//        M'[l][k] = C(l+k-1,k-1) / 2^(l+k) (k >= 1), M'[l][0] = -1/(l 2^l) (entries <= 1/2):
//        a pre-scaling, one constant Pascal-type matrix and a post-scaling (Section 4)
//   L2L  b~'_l = s^l sum_{k>=l} b~_k C(k,l) w^(k-l)
//   L2P  phi += Re sum_l b~_l xi^l
// Only the real part of the potential is needed, so the imaginary part of log(-z0) is dropped.
//
// Work decomposition.  Interaction lists of balanced trees over clustered points range from a
// few entries to thousands per box, so M2L and the near field run over the flat pair arrays of
// the lists: every warp takes a fixed chunk of consecutive pairs (sorted by target), each lane a
// contiguous sub-chunk; partial sums of equal targets are combined by a warp-segmented reduction
// and added to the target with atomics.  The near-field sums of the binary32 path are kept and
// flushed as float-float pairs, which keeps the accumulation error at the level of a few hundred
// binary32 terms.
#include <math.h>

#include <algorithm>
#include <array>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"

namespace fmm {

constexpr int PMAXC = 41;  // p <= 40

__constant__ double c_md[PMAXC][PMAXC];     // M'[l][k] in binary64
// log2(j / 128) for j = 128 .. 256 as float-float (high, low): the table of the float-float
// logarithm of the split mode's near field
__constant__ float c_lg2t[3][129];  // log2(1 + j/128) as float-float, and 1 / (1 + j/128)
// binomials C(n, k), n, k < PMAXC, in global memory: blocks copy them to shared memory (a warp
// reading many different __constant__ addresses at once would be serialised)
__device__ float g_binom_f[PMAXC * PMAXC];
__device__ double g_binom_d[PMAXC * PMAXC];

namespace {

constexpr double MIXED_TOL_FLOOR = 1e-7;  // smallest tolerance the binary32 path is asked for
constexpr int M2L_CH = 8;   // consecutive weak pairs per lane
constexpr int P2P_CH = 16;  // consecutive leaf pairs per warp
constexpr int P2P_GROUP_CH = 8;  // consecutive leaf pairs per lane group (binary32 kernel)

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

// M'[l][k] as compile-time constants for the binary32 M2L kernel, so that every product takes
// its coefficient as an immediate operand.  The binomials follow Pascal's rule in binary64, the
// same additions in the same order as the host table (exact below 2^53, identically rounded
// above), and the scaling by 2^-(l+k) is exact: the values equal the host table rounded to binary32
// bit for bit (checked when the tables are made).
template <int N, int K>
struct PascalD {
    static constexpr double v = PascalD<N - 1, K - 1>::v + PascalD<N - 1, K>::v;
};
template <int N>
struct PascalD<N, 0> {
    static constexpr double v = 1.0;
};
template <int K>
struct PascalD<0, K> {
    static constexpr double v = 0.0;
};
template <>
struct PascalD<0, 0> {
    static constexpr double v = 1.0;
};

constexpr double pow2_neg(int n)
{
    double r = 1.0;
    for (int i = 0; i < n; i++) r *= 0.5;
    return r;
}

template <int L, int K>
struct MCoef {
    static constexpr float v = (float)(PascalD<L + K - 1, K - 1>::v * pow2_neg(L + K));
};
template <int L>
struct MCoef<L, 0> {
    static constexpr float v = (float)(-1.0 / ((double)L / pow2_neg(L)));
};
template <>
struct MCoef<0, 0> {
    static constexpr float v = 0.0f;
};

// All M' coefficients as compiled, for the host to compare with its table.
template <int... I>
constexpr std::array<float, sizeof...(I)> mcoef_table(std::integer_sequence<int, I...>)
{
    return {MCoef<I / PMAXC, I % PMAXC>::v...};
}

// One term M'[O][K] x_K of row O into the partial sums of parity K & 1; zero coefficients and the
// zero imaginary part of x_0 (= a~_0, real) contribute nothing and are left out.
template <int O, int K>
__device__ __forceinline__ void m2l_term(const cx<float>* x, float (&yr)[2], float (&yi)[2])
{
    if constexpr (MCoef<O, K>::v != 0.0f) {
        yr[K & 1] = fmaf(MCoef<O, K>::v, x[K].re, yr[K & 1]);
        if constexpr (K > 0) yi[K & 1] = fmaf(MCoef<O, K>::v, x[K].im, yi[K & 1]);
    }
}

// Row O of y = M' x with immediate coefficients: even and odd k in two partial sums (two
// independent chains of dependent FMAs instead of one), added at the end.
template <int O, int... K>
__device__ __forceinline__ cx<float> m2l_row(const cx<float>* x, std::integer_sequence<int, K...>)
{
    float yr[2] = {0.f, 0.f}, yi[2] = {0.f, 0.f};
    (m2l_term<O, K>(x, yr, yi), ...);
    return {yr[0] + yr[1], yi[0] + yi[1]};
}


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


// Box geometry in the working precision.  z0 = c_a - c_b: in binary64 directly, in binary32 from
// the float-float centres so that the difference of two nearby centres keeps its relative
// accuracy.  The binary32 path never touches binary64 arithmetic (slow on GB300): radii come
// from a binary32 copy and point coordinates are binary32 offsets from their leaf centre.
template <typename T>
struct Geo;
template <>
struct Geo<double> {
    const double* cen;
    const double* rad;
    __device__ __forceinline__ cx<double> diff(int64_t a, int64_t b) const
    {
        return {cen[2 * a] - cen[2 * b], cen[2 * a + 1] - cen[2 * b + 1]};
    }
    __device__ __forceinline__ double radius(int64_t g) const { return rad[g]; }
    __device__ __forceinline__ Geo shift(int64_t b0) const { return Geo{cen + 2 * b0, rad + b0}; }
    // z - c_b for a point of leaf a (absolute coordinates)
    __device__ __forceinline__ cx<double> rel(int64_t a, int64_t b, double x, double y) const
    {
        return {x - cen[2 * b], y - cen[2 * b + 1]};
    }
    // (z - c_g) / rho_g for a point stored with absolute coordinates (0 when rho_g = 0)
    __device__ __forceinline__ cx<double> local(int64_t g, double x, double y) const
    {
        const double rho = rad[g];
        if (!(rho > 0.0)) return {0.0, 0.0};
        return {(x - cen[2 * g]) / rho, (y - cen[2 * g + 1]) / rho};
    }
};
template <>
struct Geo<float> {
    const float* hi;
    const float* lo;
    const float* rad;
    __device__ __forceinline__ cx<float> diff(int64_t a, int64_t b) const
    {
        float2 ha = *(const float2*)(hi + 2 * a), hb = *(const float2*)(hi + 2 * b);
        float2 la = *(const float2*)(lo + 2 * a), lb = *(const float2*)(lo + 2 * b);
        return {(ha.x - hb.x) + (la.x - lb.x), (ha.y - hb.y) + (la.y - lb.y)};
    }
    __device__ __forceinline__ float radius(int64_t g) const { return rad[g]; }
    __device__ __forceinline__ Geo shift(int64_t b0) const { return Geo{hi + 2 * b0, lo + 2 * b0, rad + b0}; }
    // z - c_b for a point of leaf a (stored as its offset from c_a)
    __device__ __forceinline__ cx<float> rel(int64_t a, int64_t b, float x, float y) const
    {
        const cx<float> d = diff(a, b);
        return {d.re + x, d.im + y};
    }
    // the point is stored as its offset from the centre of leaf g
    __device__ __forceinline__ cx<float> local(int64_t g, float x, float y) const
    {
        const float rho = rad[g];
        if (!(rho > 0.f)) return {0.f, 0.f};
        const float inv = 1.f / rho;
        return {x * inv, y * inv};
    }
};

__device__ __forceinline__ double log_d(double x) { return log(x); }
__device__ __forceinline__ float log_d(float x) { return logf(x); }

// Float-float accumulation (Knuth's two-sum): hi + lo holds a sum whose rounding errors are
// carried in lo instead of lost.
__device__ __forceinline__ void two_sum(float& hi, float& lo, float v)
{
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

// hi + lo += vhi + vlo on values shared between threads: the atomic addition returns the value it
// found, so the rounding error of the sum it stored is recovered exactly by a two-sum and added to
// lo with the incoming low part.
__device__ __forceinline__ void atomic_add_ff(float* hi, float* lo, float vhi, float vlo)
{
    const float old = atomicAdd(hi, vhi);
    const float s = old + vhi;
    const float bb = s - old;
    atomicAdd(lo, ((old - (s - bb)) + (vhi - bb)) + vlo);
}

__device__ __forceinline__ float lg2_fast(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <typename T>
struct Pk;  // packed point
template <>
struct alignas(32) Pk<double> {
    double x, y, q, pad;
};
template <>
struct alignas(16) Pk<float> {
    float x, y, q, pad;
};

// ---- strengths into canonical order, packed with the coordinates ----
template <typename T>
__global__ void k_pack(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ perm,
                       const double* __restrict__ q, const double* __restrict__ xs,
                       const double* __restrict__ ys, const float* __restrict__ dxf,
                       const float* __restrict__ dyf, Pk<T>* __restrict__ pk, int32_t* status)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    perm += S.p0;
    q += S.p0;
    xs += S.p0;
    ys += S.p0;
    dxf += S.p0;
    dyf += S.p0;
    pk += S.p0;
    const int64_t n = S.n;
    bool bad = false;
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)z.nb * blockDim.x) {
        double v = q[perm[i]];
        bad |= !isfinite(v);
        Pk<T> p;
        if (sizeof(T) == 8) {
            p.x = (T)xs[i];
            p.y = (T)ys[i];
        } else {
            p.x = (T)dxf[i];
            p.y = (T)dyf[i];
        }
        p.q = (T)v;
        p.pad = 0;
        pk[i] = p;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// ---- P2M: one warp per leaf, one lane per point; column sums through shared memory ----
template <typename T>
__global__ void k_p2m(Sched sc, const Inst* __restrict__ I, int P, int PS, const int32_t* __restrict__ lb,
                      const Pk<T>* __restrict__ pk, Geo<T> geo, cx<T>* __restrict__ Me)
{
    extern __shared__ unsigned char smem[];
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const int L = S.L;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    if (L < 1) return;
    lb += S.lb0;
    pk += S.p0;
    geo = geo.shift(S.b0);
    Me += S.b0 * PS;
    cx<T>* Sm = (cx<T>*)smem + (size_t)w * 33 * P;
    for (int64_t b = (int64_t)z.rank * wpb + w; b < level_size(L); b += (int64_t)z.nb * wpb) {
        const int64_t g = level_base(L) + b;
        const int32_t t0 = lb[b], t1 = lb[b + 1];
        cx<T> acc[2] = {{0, 0}, {0, 0}};
        for (int32_t tb = t0; tb < t1; tb += 32) {
            const int32_t t = tb + lane;
            T qq = 0;
            cx<T> xi_c = {0, 0};
            if (t < t1) {
                const Pk<T> p = pk[t];
                qq = p.q;
                xi_c = geo.local(g, p.x, p.y);
            }
            cx<T> pw = {qq, 0};
            for (int k = 0; k < P; k++) {
                Sm[k * 33 + lane] = pw;
                pw = cmul(pw, xi_c);
            }
            __syncwarp();
            for (int k = lane, s = 0; k < P; k += 32, s++) {
                cx<T> sum = {0, 0};
                for (int j = 0; j < 32; j++) sum = cadd(sum, Sm[k * 33 + j]);
                acc[s] = cadd(acc[s], sum);
            }
            __syncwarp();
        }
        for (int k = lane, s = 0; k < P; k += 32, s++)
            Me[g * PS + k] = k == 0 ? acc[s] : cscale(acc[s], (T)-1 / (T)k);
    }
}

// Binomial table C(n, k), n, k < P, copied to shared memory by the whole block.
template <typename T>
__device__ __forceinline__ void load_binom(T* B, int P)
{
    const T* src;
    if constexpr (sizeof(T) == 4) src = g_binom_f;
    else src = g_binom_d;
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) B[i] = src[(i / P) * PMAXC + i % P];
    __syncthreads();
}

// M2M of parent box b of level l (one warp, one lane per output coefficient): the four children's
// multipoles shifted to the parent.  B: binomial table, D: this warp's scratch of P values.  CG:
// the children's coefficients are read from L2 (__ldcg), as in the queued upward pass, where other
// blocks of the same launch wrote them.
template <typename T, bool CG>
__device__ __forceinline__ void m2m_box(int l, int64_t b, int P, int PS, const Geo<T>& geo, cx<T>* __restrict__ Me,
                                        const T* B, cx<T>* D, int lane)
{
    const int64_t g = level_base(l) + b;
    const T rp = geo.radius(g);
    cx<T> acc[2] = {{0, 0}, {0, 0}};
    for (int k = 0; k < 4; k++) {
        const int64_t cg = level_base(l + 1) + 4 * b + k;
        cx<T> wv = {0, 0};
        T s = 0;
        if (rp > 0) {
            const T ir = (T)1 / rp;
            wv = cscale(geo.diff(cg, g), ir);
            s = geo.radius(cg) * ir;
        }
        for (int j = lane; j < P; j += 32) {
            cx<T> m;
            if constexpr (!CG) {
                m = Me[cg * PS + j];
            } else if constexpr (sizeof(T) == 8) {
                const double2 v = __ldcg((const double2*)(Me + cg * PS + j));
                m = {v.x, v.y};
            } else {
                const float2 v = __ldcg((const float2*)(Me + cg * PS + j));
                m = {v.x, v.y};
            }
            D[j] = cscale(m, ipow(s, j));
        }
        __syncwarp();
        for (int o = lane, si = 0; o < P; o += 32, si++) {
            cx<T> h;
            if (o == 0) {
                h = D[0];
            } else {
                h = cscale(D[0], (T)-1 / (T)o);
                for (int j = 1; j <= o; j++) h = cfma(h, wv, cscale(D[j], B[(o - 1) * P + (j - 1)]));
            }
            acc[si] = cadd(acc[si], h);
        }
        __syncwarp();
    }
    for (int o = lane, si = 0; o < P; o += 32, si++) Me[g * PS + o] = acc[si];
}

// ---- M2M: one warp per parent, one lane per output coefficient ----
template <typename T>
__global__ void k_m2m(Sched sc, const Inst* __restrict__ I, int l, int P, int PS, Geo<T> geo, cx<T>* __restrict__ Me)
{
    extern __shared__ unsigned char smem[];
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    if (l + 1 > S.L) return;
    geo = geo.shift(S.b0);
    Me += S.b0 * PS;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    T* B = (T*)smem;
    cx<T>* D = (cx<T>*)(smem + ((P * P * sizeof(T) + 15) & ~15)) + (size_t)w * P;
    load_binom(B, P);
    for (int64_t b = (int64_t)z.rank * wpb + w; b < level_size(l); b += (int64_t)z.nb * wpb)
        m2m_box<T, false>(l, b, P, PS, geo, Me, B, D, lane);
}

// ---- the upward (M2M) and downward (L2L) passes as persistent launches over work queues ----
//
// One launch does every level of every instance.  The queue lists items (QBOX boxes of one level
// of one instance) in dependency order: the upward pass from the deepest M2M level up, the
// downward pass from level 1 down.  Blocks take items by ticket (an atomic counter), so every item
// an item waits for has been taken by a running block.  A level's items may start once the
// instance's level below (upward) or above (downward) is complete: a counter per instance and
// level counts finished items, and the first thread of the block waits for it to reach the
// level's item count.  The wait is bounded: if it gives up, the status word gets the timeout bit,
// the item's work is skipped (its counter still advances, so nothing waits on it forever) and the
// evaluation reports FMM_ERR_TIMEOUT.
template <typename T, bool CG>
__device__ __forceinline__ void l2l_child(int l, int64_t c, int P, int PS, const Geo<T>& geo, cx<T>* __restrict__ Le,
                                          float* __restrict__ L0lo, const T* Bn, cx<T>* B, int lane);

constexpr int QBOX = 16;                              // boxes per queue item
constexpr int64_t Q_SPIN_LIMIT = int64_t(1) << 21;    // tries of a dependency wait (about a second)
constexpr int QBLOCKS_PER_SM = 8;

template <typename T, bool UP>
__global__ void __launch_bounds__(128) k_pass_queue(const QItem* __restrict__ items, int nitems,
                                                    const int32_t* __restrict__ need, uint32_t* done,
                                                    uint32_t* ticket, int64_t spin_limit, int32_t* status,
                                                    const Inst* __restrict__ I, int P, int PS, Geo<T> geo0,
                                                    cx<T>* __restrict__ E0, float* __restrict__ L0lo0)
{
    extern __shared__ unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    T* Bt = (T*)smem;
    cx<T>* D = (cx<T>*)(smem + ((P * P * sizeof(T) + 15) & ~15)) + (size_t)w * P;
    load_binom(Bt, P);
    __shared__ int it_s, ok_s;
    for (;;) {
        if (threadIdx.x == 0) it_s = (int)atomicAdd(ticket, 1u);
        __syncthreads();
        const int it = it_s;
        if (it >= nitems) break;  // block-uniform
        const QItem q = items[it];
        const Inst S = I[q.inst];
        const int dep = UP ? q.level + 1 : q.level - 1;
        const bool has_dep = UP ? dep < S.L : q.level >= 2;  // the leaves come from P2M, level 1 from M2L
        if (threadIdx.x == 0) {
            int ok = 1;
            if (has_dep) {
                const int64_t slot = (int64_t)q.inst * QLEVELS + dep;
                const uint32_t want = (uint32_t)need[slot];
                int64_t spins = 0;
                while (atomicAdd(done + slot, 0u) < want) {
                    if (++spins > spin_limit) {
                        atomicOr(status, ST_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
            ok_s = ok;
        }
        __syncthreads();
        if (ok_s) {
            const Geo<T> geo = geo0.shift(S.b0);
            cx<T>* E = E0 + S.b0 * PS;
            if (UP) {
                for (int b = q.b0 + w; b < q.b0 + q.nb; b += wpb)
                    m2m_box<T, true>(q.level, b, P, PS, geo, E, Bt, D, lane);
            } else {
                float* L0 = sizeof(T) == 4 ? L0lo0 + S.b0 : nullptr;
                for (int c = 4 * q.b0 + w; c < 4 * (q.b0 + q.nb); c += wpb)
                    l2l_child<T, true>(q.level, c, P, PS, geo, E, L0, Bt, D, lane);
            }
        }
        __threadfence();  // every thread's coefficients of this item before its count
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(done + (int64_t)q.inst * QLEVELS + q.level, 1u);
    }
}

// Queue memory: items up, items down, needs up, needs down [n_inst][QLEVELS] (int32), then the
// counters cleared before each pass: done up, done down [n_inst][QLEVELS], two tickets.
struct QView {
    QItem *up, *dn;
    int32_t *need_up, *need_dn;
    uint32_t *done_up, *done_dn, *tickets;
};

QView qview(fmm_tree t)
{
    const int64_t ni = t->n_inst;
    QView v;
    v.up = (QItem*)t->qmem;
    v.dn = v.up + t->nq_up;
    v.need_up = (int32_t*)(v.dn + t->nq_dn);
    v.need_dn = v.need_up + ni * QLEVELS;
    v.done_up = (uint32_t*)(v.need_dn + ni * QLEVELS);
    v.done_dn = v.done_up + ni * QLEVELS;
    v.tickets = v.done_dn + ni * QLEVELS;
    return v;
}

template <typename T, bool UP>
int launch_pass_queue(fmm_tree t, int P, int PS, const Geo<T>& geo, cx<T>* E, float* L0lo, cudaStream_t s,
                      const int32_t* need = nullptr, int32_t* status = nullptr, int64_t spin_limit = Q_SPIN_LIMIT)
{
    const int nitems = UP ? t->nq_up : t->nq_dn;
    if (nitems == 0) return 0;
    const QView v = qview(t);
    const size_t sm = ((P * P * sizeof(T) + 15) & ~15) + 4 * P * sizeof(cx<T>);
    int dev = 0, sms = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    FMM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)std::min<int64_t>(nitems, (int64_t)sms * QBLOCKS_PER_SM);
    k_pass_queue<T, UP><<<grid, 128, sm, s>>>(UP ? v.up : v.dn, nitems, need ? need : (UP ? v.need_up : v.need_dn),
                                             UP ? v.done_up : v.done_dn, v.tickets + (UP ? 0 : 1), spin_limit,
                                             status ? status : t->status, t->dinst, P, PS, geo, E, L0lo);
    note_launch();
    FMM_LAUNCH_CHECK(UP ? "evaluate: M2M (queued)" : "evaluate: L2L (queued)");
    return 0;
}

// ---- M2L over the flat weak-pair array of all levels ----
// binary32, PI = compile-time bound on P (runtime P <= PI; coefficients beyond P are zero): the
// scaled source coefficients and the partial sums live in registers, the constant matrix is read
// from the constant bank by the unrolled contraction.
// The rows of b~ += (v^l) (M' x) for one pair, O = 0 .. PI-1 at compile time: b~_0 (with the log
// term t0) in float-float, the others scaled by vp = (2v)^O.
template <int PI, int O>
__device__ __forceinline__ void m2l_rows(const cx<float>* x, cx<float>* acc, float& lo0, cx<float> vp, cx<float> v2,
                                         float t0)
{
    if constexpr (O < PI) {
        const cx<float> y = m2l_row<O>(x, std::make_integer_sequence<int, PI>{});
        if constexpr (O == 0) {
            two_sum(acc[0].re, lo0, t0);
            two_sum(acc[0].re, lo0, y.re);
            acc[0].im += y.im;
        } else {
            acc[O] = cfma(vp, y, acc[O]);
        }
        m2l_rows<PI, O + 1>(x, acc, lo0, cmul(vp, v2), v2, t0);
    }
}

template <typename T, int PI>
__global__ void __launch_bounds__(128, (PI >= 18 && PI <= 21) ? 4 : 1) k_m2l_pairs(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                                                   int P, int PS, const int32_t* __restrict__ woff,
                                                   const int32_t* __restrict__ widx,
                                                   const int32_t* __restrict__ wrow, Geo<T> geo,
                                                   const cx<T>* __restrict__ Me, cx<T>* __restrict__ Le,
                                                   float* __restrict__ L0lo)
{
    static_assert(sizeof(T) == 4, "the binary64 M2L is k_m2l_pairs_f64");
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    if (S.L < 1) return;
    woff += S.o0;
    widx += TL.w0;
    wrow += TL.w0 >> 3;
    const int64_t wcap = TL.wcap, nbox = S.nbox;
    geo = geo.shift(S.b0);
    Me += S.b0 * PS;
    Le += S.b0 * PS;
    L0lo += S.b0;
    const int lane = threadIdx.x & 31;
    const int64_t e_begin = woff[1];
    const int64_t e_end = min((int64_t)woff[nbox], wcap);
    const int64_t warp = ((int64_t)z.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)z.nb * blockDim.x) >> 5;
    for (int64_t wb = e_begin + warp * 32 * M2L_CH; wb < e_end; wb += nwarps * 32 * M2L_CH) {
        const int64_t e0 = wb + (int64_t)lane * M2L_CH;
        const int64_t e1 = min(e0 + M2L_CH, e_end);
        // Re b_0 carries the whole far potential (large terms that cancel little): it is summed
        // in float-float, acc[0].re + lo0, and added to the box as hi/lo
        cx<T> acc[PI];
        T lo0 = 0;
#pragma unroll
        for (int j = 0; j < PI; j++) acc[j] = {0, 0};
        int64_t cur = -1;
        // targets from the row table and the offsets (entries are sorted by target)
        int64_t g = e0 < e1 ? wtarget_start(wrow, woff, e0) : 0;
        int64_t gend = woff[g + 1];
        for (int64_t e = e0; e < e1; e++) {
            while (e >= gend) gend = woff[(++g) + 1];
            if (g != cur) {
                if (cur >= 0) {
                    atomic_add_ff(&Le[cur * PS].re, &L0lo[cur], acc[0].re, lo0);
                    atomicAdd(&Le[cur * PS].im, acc[0].im);
#pragma unroll
                    for (int j = 1; j < PI; j++)
                        if (j < P) {
                            atomicAdd(&Le[cur * PS + j].re, acc[j].re);
                            atomicAdd(&Le[cur * PS + j].im, acc[j].im);
                        }
                }
#pragma unroll
                for (int j = 0; j < PI; j++) acc[j] = {0, 0};
                lo0 = 0;
                cur = g;
            }
            const int64_t sg = weak_source(g, widx[e]);
            const cx<T> z0 = geo.diff(sg, g);
            const T r2 = z0.re * z0.re + z0.im * z0.im;
            const T ir2 = __frcp_rn(r2);  // correctly rounded, as 1 / r2
            const cx<T> inv = {z0.re * ir2, -z0.im * ir2};
            const cx<T> u2 = cscale(inv, (T)-2 * geo.radius(sg)), v2 = cscale(inv, (T)2 * geo.radius(g));
            // the source's coefficients two at a time (rows are PS = P rounded up to even long)
            const float4* src4 = (const float4*)(Me + sg * PS);
            float4 q4 = src4[0];
            const T a0 = q4.x;
            cx<T> x[PI];
            x[0] = {a0, 0};
            cx<T> up = u2;
#pragma unroll
            for (int k = 1; k < PI; k++) {
                if ((k & 1) == 0) q4 = (k < P) ? src4[k >> 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                cx<T> v = {0, 0};
                if (k < P) v = cmul((k & 1) ? cx<T>{q4.z, q4.w} : cx<T>{q4.x, q4.y}, up);
                x[k] = v;
                up = cmul(up, u2);
            }
            m2l_rows<PI, 0>(x, acc, lo0, cx<float>{1.f, 0.f}, v2, a0 * 0.5f * log_d(r2));
        }
        // warp-segmented reduction of the last partial sums (targets are non-decreasing across
        // lanes; lanes without pairs carry -1 and sit at the end)
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t pkey = __shfl_down_sync(0xffffffffu, cur, off);
            const bool take = (lane + off < 32) && pkey == cur;
            const T plo = __shfl_down_sync(0xffffffffu, lo0, off);
#pragma unroll
            for (int j = 0; j < PI; j++) {
                const T pr = __shfl_down_sync(0xffffffffu, acc[j].re, off);
                const T pi = __shfl_down_sync(0xffffffffu, acc[j].im, off);
                if (take) {
                    if (j == 0) {
                        two_sum(acc[0].re, lo0, pr);
                        lo0 += plo;
                    } else {
                        acc[j].re += pr;
                    }
                    acc[j].im += pi;
                }
            }
        }
        const int64_t prev = __shfl_up_sync(0xffffffffu, cur, 1);
        if (cur >= 0 && (lane == 0 || prev != cur)) {
            atomic_add_ff(&Le[cur * PS].re, &L0lo[cur], acc[0].re, lo0);
            atomicAdd(&Le[cur * PS].im, acc[0].im);
#pragma unroll
            for (int j = 1; j < PI; j++)
                if (j < P) {
                    atomicAdd(&Le[cur * PS + j].re, acc[j].re);
                    atomicAdd(&Le[cur * PS + j].im, acc[j].im);
                }
        }
    }
}

// ---- M2L, binary64: same decomposition, runtime P, operands and partial sums in shared memory
// (one thread's column of X and A; the binary64 pipe bounds this kernel) ----
__global__ void __launch_bounds__(64) k_m2l_pairs_f64(Sched sc, const Inst* __restrict__ I,
                                                      const LInst* __restrict__ LIs, int P, int PS,
                                                      const int32_t* __restrict__ woff,
                                                      const int32_t* __restrict__ widx,
                                                      const int32_t* __restrict__ wrow, Geo<double> geo,
                                                      const cx<double>* __restrict__ Me,
                                                      cx<double>* __restrict__ Le)
{
    extern __shared__ unsigned char smem[];
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    if (S.L < 1) return;
    woff += S.o0;
    widx += TL.w0;
    wrow += TL.w0 >> 3;
    const int64_t wcap = TL.wcap, nbox = S.nbox;
    geo = geo.shift(S.b0);
    Me += S.b0 * PS;
    Le += S.b0 * PS;
    const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    cx<double>* X = (cx<double>*)smem;  // X[k * nt + tid]
    cx<double>* A = X + (size_t)P * nt;  // A[o * nt + tid]
    const int64_t e_begin = woff[1];
    const int64_t e_end = min((int64_t)woff[nbox], wcap);
    const int64_t warp = ((int64_t)z.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)z.nb * blockDim.x) >> 5;
    for (int64_t wb = e_begin + warp * 32 * M2L_CH; wb < e_end; wb += nwarps * 32 * M2L_CH) {
        const int64_t e0 = wb + (int64_t)lane * M2L_CH;
        const int64_t e1 = min(e0 + M2L_CH, e_end);
        for (int j = 0; j < P; j++) A[j * nt + tid] = {0, 0};
        int64_t cur = -1;
        int64_t g = e0 < e1 ? wtarget_start(wrow, woff, e0) : 0;
        int64_t gend = woff[g + 1];
        for (int64_t e = e0; e < e1; e++) {
            while (e >= gend) gend = woff[(++g) + 1];
            if (g != cur) {
                if (cur >= 0)
                    for (int j = 0; j < P; j++) {
                        atomicAdd(&Le[cur * PS + j].re, A[j * nt + tid].re);
                        atomicAdd(&Le[cur * PS + j].im, A[j * nt + tid].im);
                        A[j * nt + tid] = {0, 0};
                    }
                cur = g;
            }
            const int64_t sg = weak_source(g, widx[e]);
            const cx<double> z0 = geo.diff(sg, g);
            const double r2 = z0.re * z0.re + z0.im * z0.im;
            const double ir2 = 1.0 / r2;
            const cx<double> inv = {z0.re * ir2, -z0.im * ir2};
            const cx<double> u2 = cscale(inv, -2.0 * geo.radius(sg)), v2 = cscale(inv, 2.0 * geo.radius(g));
            const cx<double>* src = Me + sg * PS;
            const double a0 = src[0].re;
            X[tid] = {a0, 0};
            cx<double> up = u2;
            for (int k = 1; k < P; k++) {
                X[k * nt + tid] = cmul(src[k], up);
                up = cmul(up, u2);
            }
            cx<double> vp = {1, 0};
            for (int o = 0; o < P; o++) {
                cx<double> y = {0, 0};
                for (int k = 0; k < P; k++) {
                    const double m = c_md[o][k];
                    const cx<double> xv = X[k * nt + tid];
                    y.re += m * xv.re;
                    y.im += m * xv.im;
                }
                if (o == 0) y.re += a0 * 0.5 * log(r2);
                A[o * nt + tid] = cfma(vp, y, A[o * nt + tid]);
                vp = cmul(vp, v2);
            }
        }
        const int64_t prev = __shfl_up_sync(0xffffffffu, cur, 1);
        const bool head = cur >= 0 && (lane == 0 || prev != cur);
        for (int j = 0; j < P; j++) {
            cx<double> v = A[j * nt + tid];
            for (int off = 1; off < 32; off <<= 1) {
                const int64_t pkey = __shfl_down_sync(0xffffffffu, cur, off);
                const double pr = __shfl_down_sync(0xffffffffu, v.re, off);
                const double pi = __shfl_down_sync(0xffffffffu, v.im, off);
                if ((lane + off < 32) && pkey == cur) {
                    v.re += pr;
                    v.im += pi;
                }
            }
            if (head) {
                atomicAdd(&Le[cur * PS + j].re, v.re);
                atomicAdd(&Le[cur * PS + j].im, v.im);
            }
        }
    }
}

// L2L into child c of level l + 1 (one warp): the parent's local expansion shifted to the child
// and added to it.  Bn: binomial table, B: this warp's scratch.  CG: the parent's coefficients are
// read from L2 (__ldcg), as in the queued downward pass, where another block of the launch wrote
// them.
template <typename T, bool CG>
__device__ __forceinline__ void l2l_child(int l, int64_t c, int P, int PS, const Geo<T>& geo, cx<T>* __restrict__ Le,
                                          float* __restrict__ L0lo, const T* Bn, cx<T>* B, int lane)
{
    const int64_t cg = level_base(l + 1) + c, pg = level_base(l) + (c >> 2);
    const T rp = geo.radius(pg);
    cx<T> wv = {0, 0};
    T s = 0;
    if (rp > 0) {
        const T ir = (T)1 / rp;
        wv = cscale(geo.diff(cg, pg), ir);
        s = geo.radius(cg) * ir;
    }
    for (int j = lane; j < P; j += 32) {
        if constexpr (!CG) {
            B[j] = Le[pg * PS + j];
        } else if constexpr (sizeof(T) == 8) {
            const double2 v = __ldcg((const double2*)(Le + pg * PS + j));
            B[j] = {v.x, v.y};
        } else {
            const float2 v = __ldcg((const float2*)(Le + pg * PS + j));
            B[j] = {v.x, v.y};
        }
    }
    __syncwarp();
    for (int o = lane; o < P; o += 32) {
        if constexpr (sizeof(T) == 4) {
            if (o == 0) {
                // child b_0 = parent b_0 + sum_{k >= 1} b_k w^k, added to the child's hi/lo pair
                cx<T> h = {0, 0};
                for (int k = P - 1; k >= 1; k--) h = cfma(h, wv, B[k]);
                const cx<T> r = cmul(h, wv);
                T hi = Le[cg * PS].re, lo = L0lo[cg] + (CG ? __ldcg(L0lo + pg) : L0lo[pg]);
                two_sum(hi, lo, B[0].re);
                two_sum(hi, lo, r.re);
                const T sum = hi + lo;
                L0lo[cg] = lo - (sum - hi);
                Le[cg * PS].re = sum;
                Le[cg * PS].im += B[0].im + r.im;
                continue;
            }
        }
        cx<T> h = cscale(B[P - 1], Bn[(P - 1) * P + o]);
        for (int k = P - 2; k >= o; k--) h = cfma(h, wv, cscale(B[k], Bn[k * P + o]));
        const cx<T> r = cscale(h, ipow(s, o));
        Le[cg * PS + o] = cadd(Le[cg * PS + o], r);
    }
    __syncwarp();  // B is rewritten by the next box
}

// ---- L2L: one warp per child box of level l+1 ----
template <typename T>
__global__ void k_l2l(Sched sc, const Inst* __restrict__ I, int l, int P, int PS, Geo<T> geo, cx<T>* __restrict__ Le,
                      float* __restrict__ L0lo)
{
    extern __shared__ unsigned char smem[];
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    if (l + 1 > S.L) return;
    geo = geo.shift(S.b0);
    Le += S.b0 * PS;
    if constexpr (sizeof(T) == 4) L0lo += S.b0;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    T* Bn = (T*)smem;
    cx<T>* B = (cx<T>*)(smem + ((P * P * sizeof(T) + 15) & ~15)) + (size_t)w * P;
    load_binom(Bn, P);
    for (int64_t c = (int64_t)z.rank * wpb + w; c < level_size(l + 1); c += (int64_t)z.nb * wpb)
        l2l_child<T, false>(l, c, P, PS, geo, Le, L0lo, Bn, B, lane);
}

// ---- role exchange at the finest level (Section 4) ----
// Exchange-list entries of leaf g: xoff / xidx already offset to the instance.
struct XLists {
    const int32_t* xoff;
    const int32_t* xidx;
    const int32_t* xtgt;
};

// M2P: the multipole of source leaf sg evaluated at a point, dz = z - c_sg, w = rho_s / dz:
//   phi += a_0 log|dz| + Re sum_{k>=1} a~_k w^k
// (field: minus the derivative, -(a_0 - sum_k k a~_k w^k) / dz).
template <typename T>
__device__ __forceinline__ cx<T> m2p_w(cx<T> dz, T rho, T& inv_abs2)
{
    const T a2 = dz.re * dz.re + dz.im * dz.im;
    inv_abs2 = (T)1 / a2;
    return {rho * dz.re * inv_abs2, -rho * dz.im * inv_abs2};
}

// P2L: one warp per target leaf; the points of all its P2L sources form one stream, 32 at a
// time (lane = point), each lane's terms q log|dz| and q u^l (u = rho_t / dz) go through shared
// memory and lane l sums column l.  In scaled form b~_0 += sum q log|dz|,
// b~_l += -sum q u^l / l.  The leaf is owned by its warp: plain read-modify-write of Le.
// schedule: the leaves, WPB per block (the P2M schedule)
template <typename T>
__global__ void k_p2l(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs, int P, int PS,
                      const int32_t* __restrict__ lb, const Pk<T>* __restrict__ pk, Geo<T> geo, XLists xl,
                      cx<T>* __restrict__ Le, float* __restrict__ L0lo)
{
    extern __shared__ unsigned char smem[];
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const int L = S.L;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    if (L < 1) return;
    lb += S.lb0;
    pk += S.p0;
    geo = geo.shift(S.b0);
    Le += S.b0 * PS;
    if constexpr (sizeof(T) == 4) L0lo += S.b0;
    const int32_t* xoff = xl.xoff + S.o0;
    const int32_t* xidx = xl.xidx + LIs[z.i].s0;
    const int64_t base = level_base(L);
    cx<T>* Sm = (cx<T>*)smem + (size_t)w * 33 * P;
    for (int64_t b = (int64_t)z.rank * wpb + w; b < level_size(L); b += (int64_t)z.nb * wpb) {
        const int64_t g = base + b;
        const int32_t x0 = xoff[g], x1 = xoff[g + 1];
        if (x0 == x1) continue;
        const T rho = geo.radius(g);
        cx<T> acc[2] = {{0, 0}, {0, 0}};
        T acc0 = 0;
        for (int32_t e0 = x0; e0 < x1; e0 += 32) {
            // lane k describes entry e0 + k: its source's first point and count (0 for M2P entries)
            int32_t cnt = 0, first = 0, src = 0;
            if (e0 + lane < x1) {
                const int32_t v = xidx[e0 + lane];
                if (!(v & SWAP_M2P)) {
                    first = lb[v];
                    cnt = lb[v + 1] - first;
                    src = v;
                }
            }
            int32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int32_t excl = incl - cnt, total = __shfl_sync(0xffffffffu, incl, 31);
            for (int32_t f0 = 0; f0 < total; f0 += 32) {
                const int32_t fi = f0 + lane;
                // owner: the last lane k with excl_k <= fi (excl is non-decreasing)
                int k = 0;
#pragma unroll
                for (int st = 16; st; st >>= 1) {
                    const int cand = k + st;
                    const int32_t ec = __shfl_sync(0xffffffffu, excl, cand & 31);
                    if (cand < 32 && ec <= fi) k = cand;
                }
                const int32_t fk = __shfl_sync(0xffffffffu, first, k);
                const int32_t ek = __shfl_sync(0xffffffffu, excl, k);
                const int32_t sk = __shfl_sync(0xffffffffu, src, k);
                T qq = 0, lg = 0;
                cx<T> u = {0, 0};
                if (fi < total) {
                    const Pk<T> pt = pk[fk + (fi - ek)];
                    const cx<T> dz = geo.rel(base + sk, g, pt.x, pt.y);
                    T inv2;
                    u = m2p_w(dz, rho, inv2);
                    qq = pt.q;
                    lg = qq * (T)0.5 * log_d(dz.re * dz.re + dz.im * dz.im);
                }
                cx<T> pw = {qq, 0};
                Sm[lane] = {lg, 0};
                for (int l = 1; l < P; l++) {
                    pw = cmul(pw, u);
                    Sm[l * 33 + lane] = pw;
                }
                __syncwarp();
                for (int l = lane, s2 = 0; l < P; l += 32, s2++) {
                    cx<T> sum = {0, 0};
                    for (int j = 0; j < 32; j++) sum = cadd(sum, Sm[l * 33 + j]);
                    if (l == 0) acc0 += sum.re;
                    else acc[s2] = cadd(acc[s2], sum);
                }
                __syncwarp();
            }
        }
        cx<T>* B = Le + g * PS;
        for (int l = lane, s2 = 0; l < P; l += 32, s2++) {
            if (l == 0) {
                if constexpr (sizeof(T) == 4) {
                    float hi = B[0].re, lo = L0lo[g];
                    two_sum(hi, lo, acc0);
                    B[0].re = hi;
                    L0lo[g] = lo;
                } else {
                    B[0].re += acc0;
                }
            } else {
                B[l] = cadd(B[l], cscale(acc[s2], (T)-1 / (T)l));
            }
        }
    }
}

// M2P over the flat exchange lists (entries sorted by target leaf): lane groups of gs lanes
// (gs >= the largest leaf, up to 32) each walk runs of XCH consecutive entries; a lane takes the
// target's points gl, gl + gs, ... and accumulates the values of the run's M2P sources in
// registers (MAXPL points per lane, beyond that directly), flushing them atomically when the
// target changes.  Potential: adds a_0 log|dz| + Re sum a~_k w^k to acc_re (binary32 path:
// float-float hi/lo); field (FIELD): adds -(a_0 - sum_k k a~_k w^k) / dz to acc_re/acc_im.
constexpr int XCH = 8;
constexpr int MAXPL = 4;

template <typename T>
struct Acc2 {
    T hi;
    float lo;
};

template <typename T>
__device__ __forceinline__ void acc_add(Acc2<T>& a, T v)
{
    if constexpr (sizeof(T) == 4) two_sum(a.hi, a.lo, v);
    else a.hi += v;
}

template <typename T>
__device__ __forceinline__ void acc_flush(T* hi, float* lo, int64_t i, const Acc2<T>& a)
{
    if constexpr (sizeof(T) == 4) atomic_add_ff(hi + i, lo + i, a.hi, a.lo);
    else atomicAdd(hi + i, a.hi);
}

// schedule: the near-field schedule (blocks per instance in proportion to its near work)
template <typename T, bool FIELD>
__global__ void __launch_bounds__(256) k_m2p(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                                             int P, int PS, int gs, const int32_t* __restrict__ lb,
                                             const Pk<T>* __restrict__ pk, Geo<T> geo, XLists xl,
                                             const cx<T>* __restrict__ Me, T* __restrict__ re_hi,
                                             float* __restrict__ re_lo, T* __restrict__ im_hi,
                                             float* __restrict__ im_lo)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst T_ = LIs[z.i];
    const int L = S.L;
    if (L < 1) return;
    lb += S.lb0;
    pk += S.p0;
    geo = geo.shift(S.b0);
    Me += S.b0 * PS;
    re_hi += S.p0;
    if constexpr (sizeof(T) == 4) re_lo += S.p0;
    if (FIELD) {
        im_hi += S.p0;
        if constexpr (sizeof(T) == 4) im_lo += S.p0;
    }
    const int32_t* xidx = xl.xidx + T_.s0;
    const int32_t* xtgt = xl.xtgt + T_.s0;
    const int64_t nx = min((int64_t)xl.xoff[S.o0 + S.nbox], T_.scap);
    const int64_t base = level_base(L);
    const int lane = threadIdx.x & 31, G = 32 / gs, grp = lane / gs, gl = lane % gs;
    const int64_t wg = (int64_t)z.rank * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)z.nb * (blockDim.x >> 5);
    for (int64_t r = wg * G + grp; r * XCH < nx; r += nw * G) {
        const int64_t e1 = min(r * XCH + XCH, nx);
        int64_t cur = -1;
        int32_t t0 = 0, nt = 0;
        Acc2<T> ar[MAXPL], ai[MAXPL];
        auto flush = [&]() {
#pragma unroll
            for (int j = 0; j < MAXPL; j++) {
                const int32_t k = gl + j * gs;
                if (k < nt) {
                    acc_flush(re_hi, re_lo, t0 + k, ar[j]);
                    if (FIELD) acc_flush(im_hi, im_lo, t0 + k, ai[j]);
                }
                ar[j] = {0, 0.f};
                ai[j] = {0, 0.f};
            }
        };
#pragma unroll
        for (int j = 0; j < MAXPL; j++) {
            ar[j] = {0, 0.f};
            ai[j] = {0, 0.f};
        }
        for (int64_t e = r * XCH; e < e1; e++) {
            const int32_t v = xidx[e];
            if (!(v & SWAP_M2P)) continue;
            const int64_t g = xtgt[e];
            if (g != cur) {
                flush();
                cur = g;
                t0 = lb[g - base];
                nt = lb[g - base + 1] - t0;
            }
            const int64_t sg = base + (v & ~SWAP_M2P);
            cx<T> d = {0, 0};  // c_g - c_sg (the binary32 points are offsets from c_g)
            if constexpr (sizeof(T) == 4) d = geo.diff(g, sg);
            const T rho = geo.radius(sg);
            const cx<T>* A = Me + sg * PS;
            // the value at target point t0 + k: vr (potential or Re F), vi (Im F)
            auto eval = [&](int32_t k, T& vr, T& vi) {
                const Pk<T> p = pk[t0 + k];
                cx<T> dz;
                if constexpr (sizeof(T) == 4) dz = {d.re + p.x, d.im + p.y};
                else dz = geo.rel(g, sg, p.x, p.y);
                T inv2;
                const cx<T> w = m2p_w(dz, rho, inv2);
                cx<T> h = {0, 0};
                if (FIELD) {
                    for (int kk = P - 1; kk >= 1; kk--) h = cfma(h, w, cscale(A[kk], (T)kk));
                    const cx<T> hw = cmul(h, w);
                    const cx<T> num = {A[0].re - hw.re, -hw.im};
                    const cx<T> dv = cmul(num, cx<T>{dz.re * inv2, -dz.im * inv2});
                    vr = -dv.re;
                    vi = -dv.im;
                } else {
                    for (int kk = P - 1; kk >= 1; kk--) h = cfma(h, w, A[kk]);
                    vr = A[0].re * (T)-0.5 * log_d(inv2) + cmul(h, w).re;
                    vi = 0;
                }
            };
#pragma unroll
            for (int j = 0; j < MAXPL; j++) {
                const int32_t k = gl + j * gs;
                if (k < nt) {
                    T vr, vi;
                    eval(k, vr, vi);
                    acc_add(ar[j], vr);
                    if (FIELD) acc_add(ai[j], vi);
                }
            }
            for (int32_t k = gl + MAXPL * gs; k < nt; k += gs) {  // leaves beyond MAXPL points a lane
                T vr, vi;
                eval(k, vr, vi);
                acc_flush(re_hi, re_lo, t0 + k, Acc2<T>{vr, 0.f});
                if (FIELD) acc_flush(im_hi, im_lo, t0 + k, Acc2<T>{vi, 0.f});
            }
        }
        flush();
    }
}

// ---- L2P: one thread per point (canonical order) ----
// binary64 path: adds to the binary64 accumulator, which already holds the near field (or, in
// the split mode, the M2P values).  binary32 path: writes the binary32 far field (float-float),
// or with `add` adds to the M2P values already there; the near-field accumulators are combined
// with it at the end.
template <typename T>
__global__ void k_l2p(Sched sc, const Inst* __restrict__ I, int P, int PS, const int32_t* __restrict__ cleaf,
                      const Pk<T>* __restrict__ pk, Geo<T> geo, const cx<T>* __restrict__ Le,
                      const float* __restrict__ L0lo, T* __restrict__ far, float* __restrict__ farlo, bool add)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const int L = S.L;
    const int64_t n = S.n;
    cleaf += S.p0;
    pk += S.p0;
    far += S.p0;
    geo = geo.shift(S.b0);
    Le += S.b0 * PS;
    if constexpr (sizeof(T) == 4) {
        L0lo += S.b0;
        farlo += S.p0;
    }
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)z.nb * blockDim.x) {
        const int64_t g = level_base(L) + cleaf[i];
        const Pk<T> p = pk[i];
        const cx<T> z = geo.local(g, p.x, p.y);
        const cx<T>* B = Le + g * PS;
        if constexpr (sizeof(T) == 4) {
            cx<T> h = {0, 0};
            for (int k = P - 1; k >= 1; k--) h = cfma(h, z, B[k]);
            T hi = B[0].re, lo = L0lo[g];
            two_sum(hi, lo, cmul(h, z).re);
            if (add) {  // onto the M2P values already there
                T fh = far[i];
                float fl = farlo[i];
                two_sum(fh, fl, hi);
                hi = fh;
                lo += fl;
            }
            far[i] = hi;
            farlo[i] = lo;
        } else {
            cx<T> h = B[P - 1];
            for (int k = P - 2; k >= 0; k--) h = cfma(h, z, B[k]);
            far[i] += h.re;  // binary64: the near field is already in the accumulator
        }
    }
}

// ---- near field over the flat strong-pair array of the finest level ----
//
// Pair (target leaf, source leaf) e of the finest strong lists contributes
//     phi_i += sum_{j in source leaf, z_j != z_i} q_j log|z_i - z_j|,  i in target leaf.
// binary32 path: coordinates are offsets from the leaf centres, the target is moved into the
// source frame through the float-float centre difference once per leaf pair, and
// q_j * log2(r^2) is summed in binary32 over one source leaf, then into a float-float lane
// accumulator.  A binary32 offset carries an absolute error of about 2^-25 of the leaf-pair scale
// M, so a pair closer than M/256 (which includes j = i and coincident points) takes its squared
// distance from the binary64 coordinates; every other term then has |error| < 2^-14 in log2
// units.  binary64 path: absolute coordinates, binary64 log.  Flushes add binary64 partial sums
// to the accumulator atomically.


// Leaves of at most 32 points: groups of gs = pow2ceil(max leaf size) lanes, one lane per target;
// the G = 32/gs groups of a warp walk the warp's P2P_CH consecutive pairs round robin, each group
// one whole source leaf at a time.
// Accumulators: binary64 path acc64 (holds the far field already); binary32 path nhi/nlo, the
// float-float near-field sums in log2 units (flushed with binary32 atomics).
template <typename T>
__global__ void __launch_bounds__(256) k_p2p_small(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                                                   int gs, const int32_t* __restrict__ soff,
                                                   const int32_t* __restrict__ sidx,
                                                   const int32_t* __restrict__ stgt,
                                                   const int32_t* __restrict__ lb,
                                                   const Pk<T>* __restrict__ pk,
                                                   const double* __restrict__ xs,
                                                   const double* __restrict__ ys,
                                                   const float* __restrict__ chi,
                                                   const float* __restrict__ clo,
                                                   const float* __restrict__ rad32,
                                                   double* __restrict__ acc64, float* __restrict__ nhi,
                                                   float* __restrict__ nlo)
{
    constexpr bool F32 = sizeof(T) == 4;
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    const int L = S.L;
    if ((int64_t)S.maxleaf > gs) return;  // left to k_p2p_large
    const int64_t scap = TL.scap;
    soff += S.o0;
    sidx += TL.s0;
    stgt += TL.s0;
    lb += S.lb0;
    pk += S.p0;
    xs += S.p0;
    ys += S.p0;
    chi += 2 * S.b0;
    clo += 2 * S.b0;
    rad32 += S.b0;
    acc64 += S.p0;
    nhi += S.p0;
    nlo += S.p0;
    const int lane = threadIdx.x & 31, G = 32 / gs, grp = lane / gs, ti = lane & (gs - 1);
    const int64_t base = level_base(L);
    const int64_t e_begin = min((int64_t)soff[base], scap);
    const int64_t e_end = min((int64_t)soff[base + level_size(L)], scap);
    const int64_t warp = ((int64_t)z.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)z.nb * blockDim.x) >> 5;
    for (int64_t e0 = e_begin + warp * P2P_CH; e0 < e_end; e0 += nwarps * P2P_CH) {
        const int64_t e1 = min(e0 + P2P_CH, e_end);
        int64_t cur = -1;
        int32_t it = 0;  // canonical index of this lane's target
        bool active = false;
        T tx = 0, ty = 0;
        float hi = 0.f, lo = 0.f;  // binary32 path accumulator
        double sum64 = 0.0;        // binary64 path accumulator
        for (int64_t e = e0 + grp; e < e1; e += G) {
            const int64_t tl = stgt[e] - base;
            if (tl != cur) {
                if (active) {
                    if (F32) {
                        atomicAdd(&nhi[it], hi);
                        atomicAdd(&nlo[it], lo);
                    } else {
                        atomicAdd(&acc64[it], 0.5 * sum64);
                    }
                }
                cur = tl;
                const int32_t t0 = lb[tl], nt = lb[tl + 1] - t0;
                active = ti < nt;
                it = t0 + ti;
                hi = lo = 0.f;
                sum64 = 0.0;
                if (active) {
                    const Pk<T> p = pk[it];
                    tx = p.x;
                    ty = p.y;
                }
            }
            if (!active) continue;
            const int64_t sl = sidx[e];
            const int32_t s0 = lb[sl], ns = lb[sl + 1] - s0;
            if constexpr (F32) {
                const int64_t sg = base + sl, tg = base + tl;
                const float ox = (chi[2 * sg] - chi[2 * tg]) + (clo[2 * sg] - clo[2 * tg]);
                const float oy = (chi[2 * sg + 1] - chi[2 * tg + 1]) + (clo[2 * sg + 1] - clo[2 * tg + 1]);
                const float xt = tx - ox, yt = ty - oy;
                const float M = rad32[sg] + rad32[tg] + fabsf(ox) + fabsf(oy);
                const float tau2 = fmaxf((M * (1.f / 256.f)) * (M * (1.f / 256.f)), 1e-30f);  // > 0: r = 0 is exact
                float part = 0.f;
#pragma unroll 4
                for (int j = 0; j < ns; j++) {
                    const Pk<float> sp = pk[s0 + j];
                    const float dx = xt - sp.x, dy = yt - sp.y;
                    const float r2 = dx * dx + dy * dy;
                    if (r2 >= tau2) {
                        part += sp.q * __log2f(r2);
                    } else {
                        const double ddx = xs[it] - xs[s0 + j], ddy = ys[it] - ys[s0 + j];
                        const double r2d = ddx * ddx + ddy * ddy;
                        if (r2d >= 1e-36) part += sp.q * lg2_fast((float)r2d);
                            else if (r2d > 0.0) part += sp.q * (float)log2(r2d);
                    }
                }
                two_sum(hi, lo, part);
            } else {
                double part = 0.0;
                for (int j = 0; j < ns; j++) {
                    const Pk<double> sp = pk[s0 + j];
                    const double dx = tx - sp.x, dy = ty - sp.y;
                    const double r2 = dx * dx + dy * dy;
                    if (r2 > 0.0) part += sp.q * log(r2);
                }
                sum64 += part;
            }
        }
        if (active) {
            if (F32) {
                atomicAdd(&nhi[it], hi);
                atomicAdd(&nlo[it], lo);
            } else {
                atomicAdd(&acc64[it], 0.5 * sum64);
            }
        }
    }
}


// Sum of one target against one source leaf when some pair is closer than sqrt(tau2): the binary32
// offsets (rounded to about 2^-24 of the leaf-pair extent M) cannot resolve such a pair, so its
// squared distance is taken from the binary64 coordinates; the logarithm stays binary32, whose
// absolute error does not grow as r shrinks.  j = i and coincident points are skipped.
__device__ __forceinline__ float p2p_exact(float xt, float yt, int32_t it, const Pk<float>* __restrict__ pk,
                                           int32_t s0, int32_t ns, float tau2, const double* __restrict__ xs,
                                           const double* __restrict__ ys)
{
    float part = 0.f;
    for (int32_t j = 0; j < ns; j++) {
        if (s0 + j == it) continue;
        const Pk<float> sp = pk[s0 + j];
        const float dx = xt - sp.x, dy = yt - sp.y;
        const float r2 = dx * dx + dy * dy;
        if (r2 >= tau2) {
            part += sp.q * lg2_fast(r2);
        } else {
            const double ddx = xs[it] - xs[s0 + j], ddy = ys[it] - ys[s0 + j];
            const double r2d = ddx * ddx + ddy * ddy;
            if (r2d >= 1e-36)
                part += sp.q * lg2_fast((float)r2d);
            else if (r2d > 0.0)  // below the binary32 normal range
                part += sp.q * (float)log2(r2d);
        }
    }
    return part;
}

// binary32 near field for leaves of at most 64 points.  Groups of gsl lanes work on one leaf pair,
// each lane on NT targets (t0 + li + k gsl, k < NT), so a warp holds 32 / gsl leaf pairs at once
// and every source load serves NT pair evaluations; each group walks its own run of consecutive
// leaf pairs and flushes its sums when the target leaf changes.  More targets per lane spread the
// per-leaf-pair set-up (geometry loads, scale, flushes) over more pairs.  The main loop has no
// branch: it keeps the smallest r^2 it met and, for the rare lane whose minimum falls below the
// exactness threshold, the leaf pair is redone by the exact path.
template <int NT>
__global__ void __launch_bounds__(256) k_p2p_f32(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                                                 const int32_t* __restrict__ soff,
                                                 const int32_t* __restrict__ sidx,
                                                 const int32_t* __restrict__ stgt,
                                                 const int32_t* __restrict__ lb,
                                                 const Pk<float>* __restrict__ pk,
                                                 const double* __restrict__ xs,
                                                 const double* __restrict__ ys,
                                                 const float* __restrict__ chi,
                                                 const float* __restrict__ clo,
                                                 const float* __restrict__ rad32,
                                                 float* __restrict__ nhi, float* __restrict__ nlo)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    const int L = S.L;
    const int64_t scap = TL.scap;
    soff += S.o0;
    sidx += TL.s0;
    stgt += TL.s0;
    lb += S.lb0;
    pk += S.p0;
    xs += S.p0;
    ys += S.p0;
    chi += 2 * S.b0;
    clo += 2 * S.b0;
    rad32 += S.b0;
    nhi += S.p0;
    nlo += S.p0;
    // groups of gsl lanes, NT targets per lane: gsl = pow2ceil(largest leaf of this instance) / NT
    const int64_t maxleaf = (int64_t)S.maxleaf;
    if (maxleaf > 64) return;  // left to k_p2p_large
    int gsl = 1;
    while (NT * gsl < maxleaf) gsl <<= 1;
    const int lane = threadIdx.x & 31, G = 32 / gsl, grp = lane / gsl, li = lane - grp * gsl;
    const int32_t base = (int32_t)level_base(L);
    const int64_t e_begin = min((int64_t)soff[base], scap);
    const int64_t e_end = min((int64_t)soff[base + level_size(L)], scap);
    const int64_t warp = ((int64_t)z.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)z.nb * blockDim.x) >> 5;
    // each group takes P2P_GROUP_CH consecutive leaf pairs of the warp's chunk, so its target leaf
    // changes (and its partial sums are flushed) only where the list moves to the next target
    const int64_t wch = (int64_t)G * P2P_GROUP_CH;
    for (int64_t w0 = e_begin + warp * wch; w0 < e_end; w0 += nwarps * wch) {
        const int64_t e0 = w0 + (int64_t)grp * P2P_GROUP_CH;
        const int64_t e1 = min(e0 + P2P_GROUP_CH, e_end);
        int32_t cur = -1, t0 = 0, nt = 0;
        float tx[NT], ty[NT], tq[NT], hi[NT], lo[NT];
#pragma unroll
        for (int k = 0; k < NT; k++) tx[k] = ty[k] = tq[k] = hi[k] = lo[k] = 0.f;
        float2 tch = make_float2(0.f, 0.f), tcl = tch;  // the target leaf's float-float centre
        float trad = 0.f;                                // and binary32 radius
        auto flush = [&]() {
#pragma unroll
            for (int k = 0; k < NT; k++)
                if (li + k * gsl < nt) {
                    atomicAdd(&nhi[t0 + li + k * gsl], hi[k]);
                    atomicAdd(&nlo[t0 + li + k * gsl], lo[k]);
                }
        };
        for (int64_t e = e0; e < e1; e++) {
            const int32_t tl = stgt[e] - base;
            if (tl != cur) {
                if (cur >= 0) flush();
                cur = tl;
                t0 = lb[tl];
                nt = lb[tl + 1] - t0;
                tch = *(const float2*)(chi + 2 * (base + tl));
                tcl = *(const float2*)(clo + 2 * (base + tl));
                trad = rad32[base + tl];
#pragma unroll
                for (int k = 0; k < NT; k++) {
                    hi[k] = lo[k] = 0.f;
                    if (li + k * gsl < nt) {
                        const Pk<float> p = pk[t0 + li + k * gsl];
                        tx[k] = p.x;
                        ty[k] = p.y;
                        tq[k] = p.q;
                    }
                }
            }
            if (li >= nt) continue;  // target k > 0 valid implies target 0 valid
            const int32_t sl = sidx[e];
            const int32_t s0 = lb[sl], ns = lb[sl + 1] - s0;
            const int32_t sg = base + sl;
            const float2 sch = *(const float2*)(chi + 2 * sg), scl = *(const float2*)(clo + 2 * sg);
            const float ox = (sch.x - tch.x) + (scl.x - tcl.x);
            const float oy = (sch.y - tch.y) + (scl.y - tcl.y);
            const float M = rad32[sg] + trad + fabsf(ox) + fabsf(oy);
            const float tau2 = fmaxf((M * (1.f / 256.f)) * (M * (1.f / 256.f)), 1e-30f);
            // logs are taken of r^2 / 2^e, 2^e the power of two at or below M^2 (near 1 for most
            // pairs), and e times the sources' strength is added once per leaf pair: the running
            // sums stay small, and the scaling and its logarithm are exact
            const float M2 = M * M;
            const bool scaled = M2 > 1e-30f && M2 < 1e30f;
            const int ex = scaled ? (int)((__float_as_uint(M2) >> 23) & 0xff) - 127 : 0;
            const float s2 = __uint_as_float((uint32_t)(127 - ex) << 23);  // 2^-ex
            const float c2 = (float)ex;
            float xa[NT], ya[NT], pa[NT], ma[NT];
#pragma unroll
            for (int k = 0; k < NT; k++) {
                xa[k] = tx[k] - ox;
                ya[k] = ty[k] - oy;
                pa[k] = 0.f;
                ma[k] = 3.0e38f;
            }
            float qs = 0.f;
            const Pk<float>* src = pk + s0;
            if (sl != tl) {
#pragma unroll 16 / NT
                for (int32_t j = 0; j < ns; j++) {
                    const float4 sp = *(const float4*)(src + j);  // x, y, q in one load
                    qs += sp.z;
#pragma unroll
                    for (int k = 0; k < NT; k++) {
                        const float dx = xa[k] - sp.x, dy = ya[k] - sp.y;
                        const float r = dx * dx + dy * dy;
                        ma[k] = fminf(ma[k], r);
                        pa[k] += sp.z * lg2_fast(r * s2);
                    }
                }
#pragma unroll
                for (int k = 0; k < NT; k++) pa[k] += c2 * qs;
            } else {
                // the leaf with itself: a point meets itself once; that term is left out
#pragma unroll 16 / NT
                for (int32_t j = 0; j < ns; j++) {
                    const float4 sp = *(const float4*)(src + j);
                    qs += sp.z;
#pragma unroll
                    for (int k = 0; k < NT; k++) {
                        const bool self = j == li + k * gsl;
                        const float dx = xa[k] - sp.x, dy = ya[k] - sp.y;
                        const float r = self ? 3.0e38f : dx * dx + dy * dy;
                        ma[k] = fminf(ma[k], r);
                        pa[k] += self ? 0.f : sp.z * lg2_fast(r * s2);
                    }
                }
#pragma unroll
                for (int k = 0; k < NT; k++) pa[k] += c2 * (qs - tq[k]);
            }
#pragma unroll
            for (int k = 0; k < NT; k++)
                if (li + k * gsl < nt) {
                    if (ma[k] < tau2) pa[k] = p2p_exact(xa[k], ya[k], t0 + li + k * gsl, pk, s0, ns, tau2, xs, ys);
                    two_sum(hi[k], lo[k], pa[k]);
                }
        }
        flush();
    }
}

// Leaves of more than small_leaf points.  The work of one leaf pair is cut into items (block of
// 32 targets, block of sources), and the items of all pairs are numbered by a scan, so one large
// pair spreads over many warps: the uniform-grid mesh can put most points into a few leaves.
// One lane per target; one flush per item.
constexpr int P2P_SCH = 1024;         // sources per item (coarser for very large leaves)
constexpr int64_t P2P_ITEMS_MAX = int64_t(1) << 20;  // items of one pair at most

// Source blocks of a pair: about P2P_SCH sources each, at most P2P_ITEMS_MAX items per pair.
__device__ __forceinline__ int32_t p2p_src_blocks(int32_t nt, int32_t ns)
{
    const int64_t ntc = (nt + 31) / 32;
    int64_t nsc = (ns + P2P_SCH - 1) / P2P_SCH;
    if (ntc * nsc > P2P_ITEMS_MAX) nsc = max((int64_t)1, P2P_ITEMS_MAX / ntc);
    return (int32_t)nsc;
}

// Work items [v0, v1) of the near field's item numbering, shared out to warps in contiguous
// ranges: warp w of nwarps takes [va, vb) and the pair e owning va (the last e with pos[e] <= va;
// pairs without items share pos).  Inside the range the owning pair only moves forward, so one
// search per warp replaces one per item.
struct ItemRange {
    int64_t va, vb, e;
};
__device__ __forceinline__ ItemRange item_range(const int32_t* __restrict__ pos, int64_t e_begin, int64_t e_end,
                                                int64_t v0, int64_t v1, int64_t warp, int64_t nwarps)
{
    ItemRange r;
    const int64_t per = (v1 - v0 + nwarps - 1) / nwarps;
    r.va = min(v0 + warp * per, v1);
    r.vb = min(r.va + per, v1);
    int64_t lo = e_begin, hi = e_end - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (pos[mid] <= r.va) lo = mid;
        else hi = mid - 1;
    }
    r.e = lo;
    return r;
}

// items[T.s0 + e] for every position e of an instance's strong array (0 outside the finest
// level's pairs and for instances left to the leaf-pair kernels); schedule: near field
__global__ void __launch_bounds__(256) k_p2p_items(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                                                   int small_leaf, const int32_t* __restrict__ soff,
                                                   const int32_t* __restrict__ sidx,
                                                   const int32_t* __restrict__ stgt,
                                                   const int32_t* __restrict__ lb, int32_t* __restrict__ items,
                                                   unsigned long long* total)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    soff += S.o0;
    sidx += TL.s0;
    stgt += TL.s0;
    lb += S.lb0;
    items += TL.s0;
    const bool mine = S.maxleaf > small_leaf;
    const int64_t base = level_base(S.L);
    const int64_t e_begin = min((int64_t)soff[base], TL.scap);
    const int64_t e_end = min((int64_t)soff[base + level_size(S.L)], TL.scap);
    unsigned long long sum = 0;
    for (int64_t e = (int64_t)z.rank * blockDim.x + threadIdx.x; e < TL.scap; e += (int64_t)z.nb * blockDim.x) {
        int32_t v = 0;
        if (mine && e >= e_begin && e < e_end) {
            const int64_t tl = stgt[e] - base, sl = sidx[e];
            const int32_t nt = lb[tl + 1] - lb[tl], ns = lb[sl + 1] - lb[sl];
            v = nt > 0 && ns > 0 ? (int32_t)((nt + 31) / 32) * p2p_src_blocks(nt, ns) : 0;
        }
        items[e] = v;
        sum += (unsigned long long)v;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(total, sum);  // all items: must fit the int32 scan
}

// schedule: near field; pos = exclusive scan of items over all instances' strong arrays
template <typename T>
__global__ void __launch_bounds__(256) k_p2p_large(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                                                   int small_leaf, const int32_t* __restrict__ soff,
                                                   const int32_t* __restrict__ sidx,
                                                   const int32_t* __restrict__ stgt,
                                                   const int32_t* __restrict__ lb,
                                                   const int32_t* __restrict__ pos,
                                                   const unsigned long long* __restrict__ total,
                                                   int32_t* status,
                                                   const Pk<T>* __restrict__ pk,
                                                   const double* __restrict__ xs,
                                                   const double* __restrict__ ys,
                                                   const float* __restrict__ chi,
                                                   const float* __restrict__ clo,
                                                   const float* __restrict__ rad32,
                                                   double* __restrict__ acc64, float* __restrict__ nhi,
                                                   float* __restrict__ nlo)
{
    constexpr bool F32 = sizeof(T) == 4;
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    const int L = S.L;
    if ((int64_t)S.maxleaf <= small_leaf) return;  // done by the leaf-pair kernel
    if (*total > (unsigned long long)INT32_MAX) {  // the item numbering did not fit
        if (threadIdx.x == 0) atomicOr(status, ST_ARG);
        return;
    }
    const int64_t scap = TL.scap;
    soff += S.o0;
    sidx += TL.s0;
    stgt += TL.s0;
    pos += TL.s0;
    lb += S.lb0;
    pk += S.p0;
    xs += S.p0;
    ys += S.p0;
    chi += 2 * S.b0;
    clo += 2 * S.b0;
    rad32 += S.b0;
    acc64 += S.p0;
    nhi += S.p0;
    nlo += S.p0;
    const int lane = threadIdx.x & 31;
    const int64_t base = level_base(L);
    const int64_t e_begin = min((int64_t)soff[base], scap);
    const int64_t e_end = min((int64_t)soff[base + level_size(L)], scap);
    if (e_end <= e_begin) return;
    const int64_t v0 = pos[e_begin], v1 = pos[e_end];
    const int64_t warp = ((int64_t)z.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)z.nb * blockDim.x) >> 5;
    const ItemRange rg = item_range(pos, e_begin, e_end, v0, v1, warp, nwarps);
    int64_t e = rg.e;
    for (int64_t v = rg.va; v < rg.vb; v++) {
        while (e + 1 < e_end && pos[e + 1] <= v) e++;  // the pair owning item v
        const int64_t tl = stgt[e] - base, sl = sidx[e];
        const int32_t t0 = lb[tl], nt = lb[tl + 1] - t0, s0 = lb[sl], ns = lb[sl + 1] - s0;
        const int32_t nsc = p2p_src_blocks(nt, ns), ntc = (nt + 31) / 32;
        const int32_t local = (int32_t)(v - pos[e]);
        const int32_t tc = local % ntc, scb = local / ntc;
        const int32_t slen = (ns + nsc - 1) / nsc;
        const int32_t jb0 = scb * slen, jb1 = min(ns, jb0 + slen);
        const int32_t it = t0 + tc * 32 + lane;
        if (tc * 32 + lane >= nt) continue;
        const Pk<T> p = pk[it];
        if constexpr (F32) {
            const int64_t sg = base + sl, tg = base + tl;
            const float ox = (chi[2 * sg] - chi[2 * tg]) + (clo[2 * sg] - clo[2 * tg]);
            const float oy = (chi[2 * sg + 1] - chi[2 * tg + 1]) + (clo[2 * sg + 1] - clo[2 * tg + 1]);
            const float M = rad32[sg] + rad32[tg] + fabsf(ox) + fabsf(oy);
            const float tau2 = fmaxf((M * (1.f / 256.f)) * (M * (1.f / 256.f)), 1e-30f);  // > 0: r = 0 is exact
            const float xt = p.x - ox, yt = p.y - oy;
            float hi = 0.f, lo2 = 0.f;
            for (int32_t jb = jb0; jb < jb1; jb += 32) {
                float part = 0.f;
                const int32_t je = min(jb1, jb + 32);
                for (int32_t j = jb; j < je; j++) {
                    const Pk<float> sp = pk[s0 + j];
                    const float dx = xt - sp.x, dy = yt - sp.y;
                    const float r2 = dx * dx + dy * dy;
                    if (r2 >= tau2) {
                        part += sp.q * __log2f(r2);
                    } else {
                        const double ddx = xs[it] - xs[s0 + j], ddy = ys[it] - ys[s0 + j];
                        const double r2d = ddx * ddx + ddy * ddy;
                        if (r2d >= 1e-36) part += sp.q * lg2_fast((float)r2d);
                        else if (r2d > 0.0) part += sp.q * (float)log2(r2d);
                    }
                }
                two_sum(hi, lo2, part);
            }
            atomic_add_ff(&nhi[it], &nlo[it], hi, lo2);  // many items may add to one target
        } else {
            double part = 0.0;
            for (int32_t j = jb0; j < jb1; j++) {
                const Pk<double> sp = pk[s0 + j];
                const double dx = p.x - sp.x, dy = p.y - sp.y;
                const double r2 = dx * dx + dy * dy;
                if (r2 > 0.0) part += sp.q * log(r2);
            }
            atomicAdd(&acc64[it], 0.5 * part);
        }
    }
}

// ---- float-float near field (split mode) ------------------------------------------------------
//
// Pairs of binary32 numbers (hi + lo, |lo| <= half an ulp of hi) carry about 48 bits; the
// operations are the error-free transformations of Knuth (two-sum) and Dekker (two-product, with
// the fused multiply-add), as in the double-double literature.  Each near-field term q_j log2 r^2
// is formed in float-float from float-float coordinate offsets (each point relative to its leaf
// centre, the leaf-pair offset from the binary64 centres), so its error is about 2^-46 of its
// size, and the sums are float-float too.
struct ff {
    float h, l;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_quick(float a, float b)  // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return ff_quick(s.h, s.l);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p) + (a.h * b.l + a.l * b.h);
    return ff_quick(p, e);
}
__device__ __forceinline__ ff ff_sq(ff a)
{
    const float p = a.h * a.h;
    const float e = fmaf(a.h, a.h, -p) + 2.f * a.h * a.l;
    return ff_quick(p, e);
}
__device__ __forceinline__ ff ff_split(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

// log2 of a positive float-float a (a.h a normal binary32), table-driven (Tang's method): with
// a = 2^e m (1 <= m < 2) and F = j / 128 the nearest table point, log2 a = e + log2 F +
// log2(1 + r), r = (m - F + a.l / 2^e) / F, |r| <= 2^-8; log(1 + r) by its series to r^5 (the
// first terms in float-float, the rest in binary32), times 1/ln 2 in float-float.
// The table is read at 129 different places across a warp: in shared memory (tab, a copy of
// c_lg2t) those reads take one pass; the constant bank serialises them.
__device__ __forceinline__ ff ff_log2(ff a, const float (*tab)[129])
{
    const uint32_t bits = __float_as_uint(a.h);
    const int e = (int)(bits >> 23) - 127;
    const float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);  // [1, 2)
    const int j = __float2int_rn((m - 1.f) * 128.f);                     // 0 .. 128
    const float F = 1.f + (float)j * (1.f / 128.f);
    const float invF = tab[2][j];  // 1.f / F, correctly rounded
    const ff u = ff_two_sum(m - F, ldexpf(a.l, -e));  // m - F is exact
    const float rh = u.h * invF;
    const float rl = (fmaf(-rh, F, u.h) + u.l) * invF;
    const ff r = ff_quick(rh, rl);
    const ff r2 = ff_sq(r);
    const float t3 = r2.h * rh * (1.f / 3.f - 0.25f * rh + 0.2f * r2.h);  // r^3/3 - r^4/4 + r^5/5
    ff L = ff_add(r, ff{-0.5f * r2.h, -0.5f * r2.l});
    L = ff_add(L, ff{t3, 0.f});
    const ff inv_ln2 = {1.44269502163f, 1.92596299e-8f};  // 1/ln 2 as float-float
    L = ff_mul(L, inv_ln2);
    const ff T = {tab[0][j], tab[1][j]};
    return ff_add(ff_add(ff{(float)e, 0.f}, T), L);
}

// Points of the float-float near field: offsets from their leaf's centre and strengths, each as
// float-float (canonical order).  schedule: points
__global__ void k_pack_ff(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ perm,
                          const double* __restrict__ q, const double* __restrict__ xs, const double* __restrict__ ys,
                          const int32_t* __restrict__ cleaf, const double* __restrict__ cen, float4* __restrict__ pk)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    perm += S.p0;
    q += S.p0;
    xs += S.p0;
    ys += S.p0;
    cleaf += S.p0;
    cen += 2 * S.b0;
    pk += 2 * S.p0;
    const int64_t lbase = level_base(S.L);
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x) {
        const int64_t g = lbase + cleaf[i];
        const ff x = ff_split(xs[i] - cen[2 * g]), y = ff_split(ys[i] - cen[2 * g + 1]);
        const ff w = ff_split(q[perm[i]]);
        pk[2 * i] = make_float4(x.h, x.l, y.h, y.l);
        pk[2 * i + 1] = make_float4(w.h, w.l, 0.f, 0.f);
    }
}

// Near field in float-float: the work items of k_p2p_items (leaf pair, 32 targets, a block of
// sources), a warp per item and a lane per target; the sum of q_j log2 r^2 over the item's sources
// goes to the target's float-float accumulator (nhi, nlo) with the exact two-sum atomic.
// Coincident points (r = 0, among them j = i) are skipped.  schedule: near field
__global__ void __launch_bounds__(256) k_p2p_ff(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                                                const int32_t* __restrict__ soff, const int32_t* __restrict__ sidx,
                                                const int32_t* __restrict__ stgt, const int32_t* __restrict__ lb,
                                                const int32_t* __restrict__ pos,
                                                const unsigned long long* __restrict__ total, int32_t* status,
                                                const float4* __restrict__ pk, const double* __restrict__ cen,
                                                float* __restrict__ nhi, float* __restrict__ nlo)
{
    __shared__ float tab[3][129];
    for (int i = threadIdx.x; i < 3 * 129; i += blockDim.x) (&tab[0][0])[i] = (&c_lg2t[0][0])[i];
    __syncthreads();
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    const int L = S.L;
    if (*total > (unsigned long long)INT32_MAX) {  // the item numbering did not fit
        if (threadIdx.x == 0) atomicOr(status, ST_ARG);
        return;
    }
    const int64_t scap = TL.scap;
    soff += S.o0;
    sidx += TL.s0;
    stgt += TL.s0;
    pos += TL.s0;
    lb += S.lb0;
    pk += 2 * S.p0;
    cen += 2 * S.b0;
    nhi += S.p0;
    nlo += S.p0;
    const int lane = threadIdx.x & 31;
    const int64_t base = level_base(L);
    const int64_t e_begin = min((int64_t)soff[base], scap);
    const int64_t e_end = min((int64_t)soff[base + level_size(L)], scap);
    if (e_end <= e_begin) return;
    const int64_t v0 = pos[e_begin], v1 = pos[e_end];
    const int64_t warp = ((int64_t)z.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)z.nb * blockDim.x) >> 5;
    const ItemRange rg = item_range(pos, e_begin, e_end, v0, v1, warp, nwarps);
    int64_t e = rg.e;
    for (int64_t v = rg.va; v < rg.vb; v++) {
        while (e + 1 < e_end && pos[e + 1] <= v) e++;  // the pair owning item v
        const int64_t tl = stgt[e] - base, sl = sidx[e];
        const int32_t t0 = lb[tl], nt = lb[tl + 1] - t0, s0 = lb[sl], ns = lb[sl + 1] - s0;
        const int32_t nsc = p2p_src_blocks(nt, ns), ntc = (nt + 31) / 32;
        const int32_t local = (int32_t)(v - pos[e]);
        const int32_t tc = local % ntc, scb = local / ntc;
        const int32_t slen = (ns + nsc - 1) / nsc;
        const int32_t jb0 = scb * slen, jb1 = min(ns, jb0 + slen);
        const int32_t it = t0 + tc * 32 + lane;
        if (tc * 32 + lane >= nt) continue;
        // the target relative to the source leaf's centre: its offset plus (c_t - c_s)
        const int64_t tg = base + tl, sg = base + sl;
        const float4 tp = pk[2 * it];
        const ff xt = ff_add(ff{tp.x, tp.y}, ff_split(cen[2 * tg] - cen[2 * sg]));
        const ff yt = ff_add(ff{tp.z, tp.w}, ff_split(cen[2 * tg + 1] - cen[2 * sg + 1]));
        ff acc = {0.f, 0.f};
        for (int32_t jj = jb0; jj < jb1; jj++) {
            const float4 sp = pk[2 * (s0 + jj)];
            const float4 sq = pk[2 * (s0 + jj) + 1];
            const ff dx = ff_add(xt, ff{-sp.x, -sp.y}), dy = ff_add(yt, ff{-sp.z, -sp.w});
            const ff r2 = ff_add(ff_sq(dx), ff_sq(dy));
            if (!(r2.h > 0.f)) continue;  // coincident points, j = i among them
            ff lg;
            if (r2.h >= 1e-30f) {
                lg = ff_log2(r2, tab);
            } else {  // below the binary32 normal range of the table method: binary64
                lg = ff_split(log2((double)r2.h + (double)r2.l));
            }
            acc = ff_add(acc, ff_mul(ff{sq.x, sq.y}, lg));
        }
        atomic_add_ff(&nhi[it], &nlo[it], acc.h, acc.l);  // many items may add to one target
    }
}

// ---- float-float role exchange (split mode) ---------------------------------------------------
//
// P2L and M2P of the exchange lists are point work of the finest level, like the near field, and
// in binary64 they cost as much as the near field did (binary64 arithmetic runs at 1/73 of the
// binary32 FMA rate here).  In the split mode they run in float-float: complex products and sums
// whose low parts are rounded once per operation keep about 2^-44 of each term; the expansions
// stay binary64 in memory (M2P reads a float-float copy of the multipole coefficients, P2L adds
// its float-float sums into the binary64 local expansions).
struct cff {
    ff re, im;
};

// a.h b.h = p + e exactly (Dekker's product with the fused multiply-add), the cross terms of the
// low parts added into e
__device__ __forceinline__ float ff_prod(ff a, ff b, float& e)
{
    const float p = a.h * b.h;
    e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return p;
}

// x y - u v + c: the two leading products and c.h summed with exact two-sums, every low-order
// part added once at the end; the error is about 2^-46 of max(|x y|, |u v|, |c|)
__device__ __forceinline__ ff ff_dot2(ff x, ff y, ff u, ff v, ff c)
{
    float e1, e2;
    const float p1 = ff_prod(x, y, e1), p2 = ff_prod(u, v, e2);
    const ff s = ff_two_sum(p1, -p2);
    const ff s2 = ff_two_sum(s.h, c.h);
    return ff_quick(s2.h, ((s.l + s2.l) + (e1 - e2)) + c.l);
}

// x y - u v
__device__ __forceinline__ ff ff_dot2(ff x, ff y, ff u, ff v)
{
    float e1, e2;
    const float p1 = ff_prod(x, y, e1), p2 = ff_prod(u, v, e2);
    const ff s = ff_two_sum(p1, -p2);
    return ff_quick(s.h, s.l + (e1 - e2));
}

// h w + a and h w (complex)
__device__ __forceinline__ cff cff_fma(const cff& h, const cff& w, const cff& a)
{
    return {ff_dot2(h.re, w.re, h.im, w.im, a.re), ff_dot2(h.re, w.im, ff{-h.im.h, -h.im.l}, w.re, a.im)};
}
__device__ __forceinline__ cff cff_mul(const cff& h, const cff& w)
{
    return {ff_dot2(h.re, w.re, h.im, w.im), ff_dot2(h.re, w.im, ff{-h.im.h, -h.im.l}, w.re)};
}

__device__ __forceinline__ cff cff_add(const cff& a, const cff& b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }

// a / b: the quotient of the leading parts, corrected once by the remainder a - q b
__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    const float ib = __frcp_rn(b.h);
    const float q1 = a.h * ib;
    float e;
    const float p = ff_prod(ff{q1, 0.f}, b, e);
    const float r = ((a.h - p) - e) + a.l;
    return ff_quick(q1, r * ib);
}

// log2 of a positive float-float r^2: the table method inside the binary32 normal range (far from
// its ends), binary64 outside it
__device__ __forceinline__ ff ff_log2_any(ff a, const float (*tab)[129])
{
    if (a.h >= 1e-30f && a.h <= 1e30f) return ff_log2(a, tab);
    return ff_split(log2((double)a.h + (double)a.l));
}

// rho conj(dz) / |dz|^2 (= rho / dz) and log|dz| of the offset dz = (dx, dy), float-float
__device__ __forceinline__ void ff_inv_log(ff dx, ff dy, ff rho, ff ln2h, cff& w, ff& lg, const float (*tab)[129])
{
    const ff r2 = ff_add(ff_sq(dx), ff_sq(dy));
    const ff s = ff_div(rho, r2);
    w = {ff_mul(s, dx), ff_mul(s, ff{-dy.h, -dy.l})};
    lg = ff_mul(ff_log2_any(r2, tab), ln2h);  // log|dz| = (ln 2 / 2) log2 |dz|^2
}

// The multipole coefficients as float-float (re.h, re.l, im.h, im.l), same layout as the binary64
// ones.  count = boxes x PS.
__global__ void k_coeffs_ff(const double2* __restrict__ Me, int64_t count, float4* __restrict__ Mff)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = Me[i];
        const ff re = ff_split(a.x), im = ff_split(a.y);
        Mff[i] = make_float4(re.h, re.l, im.h, im.l);
    }
}

// Split-mode M2P (potentials): the walk of k_m2p over the flat exchange lists (runs of XCH
// entries per lane group of gs lanes, a lane's points gl, gl + gs, ... of the target leaf), each
// value in float-float: dz = the point's float-float offset from its leaf centre plus the binary64
// centre difference c_g - c_s, w = rho_s / dz, Horner over the source's float-float coefficients
// (the lane's points share each coefficient load), a~_0 log|dz| + Re sum_k a~_k w^k.  A lane sums
// its points' values over the run's entries of one target in float-float and adds them to the
// binary64 accumulator when the target changes.  schedule: the near-field schedule
__global__ void __launch_bounds__(256) k_m2p_ff(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs,
                                                int P, int PS, int gs, const int32_t* __restrict__ lb,
                                                const float4* __restrict__ pk, const double* __restrict__ cen,
                                                const double* __restrict__ rad, XLists xl,
                                                const float4* __restrict__ Mff, double* __restrict__ acc)
{
    __shared__ float tab[3][129];  // the logarithm's table (see ff_log2)
    for (int i = threadIdx.x; i < 3 * 129; i += blockDim.x) (&tab[0][0])[i] = (&c_lg2t[0][0])[i];
    __syncthreads();
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst T_ = LIs[z.i];
    const int L = S.L;
    if (L < 1) return;
    lb += S.lb0;
    pk += 2 * S.p0;
    cen += 2 * S.b0;
    rad += S.b0;
    Mff += S.b0 * PS;
    acc += S.p0;
    const int32_t* xidx = xl.xidx + T_.s0;
    const int32_t* xtgt = xl.xtgt + T_.s0;
    const int64_t nx = min((int64_t)xl.xoff[S.o0 + S.nbox], T_.scap);
    const int64_t base = level_base(L);
    const ff ln2h = ff_split(0.34657359027997264);  // ln(2) / 2
    const int lane = threadIdx.x & 31, G = 32 / gs, grp = lane / gs, gl = lane % gs;
    const int64_t wg = (int64_t)z.rank * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)z.nb * (blockDim.x >> 5);
    for (int64_t r = wg * G + grp; r * XCH < nx; r += nw * G) {
        const int64_t e1 = min(r * XCH + XCH, nx);
        int64_t cur = -1;
        int32_t t0 = 0, nt = 0;
        ff ar[MAXPL];
#pragma unroll
        for (int j = 0; j < MAXPL; j++) ar[j] = {0.f, 0.f};
        auto flush = [&]() {
#pragma unroll
            for (int j = 0; j < MAXPL; j++) {
                const int32_t k = gl + j * gs;
                if (k < nt) atomicAdd(acc + t0 + k, (double)ar[j].h + (double)ar[j].l);
                ar[j] = {0.f, 0.f};
            }
        };
        for (int64_t e = r * XCH; e < e1; e++) {
            const int32_t v = xidx[e];
            if (!(v & SWAP_M2P)) continue;
            const int64_t g = xtgt[e];
            if (g != cur) {
                flush();
                cur = g;
                t0 = lb[g - base];
                nt = lb[g - base + 1] - t0;
            }
            const int64_t sg = base + (v & ~SWAP_M2P);
            const ff dcx = ff_split(cen[2 * g] - cen[2 * sg]), dcy = ff_split(cen[2 * g + 1] - cen[2 * sg + 1]);
            const ff rho = ff_split(rad[sg]);
            const float4* A = Mff + sg * PS;
            const float4 a0 = A[0];
            // the lane's first MAXPL points together
            cff w[MAXPL], h[MAXPL];
            ff lg[MAXPL];
#pragma unroll
            for (int j = 0; j < MAXPL; j++) {
                h[j] = {{0.f, 0.f}, {0.f, 0.f}};
                w[j] = h[j];
                lg[j] = {0.f, 0.f};
                const int32_t k = gl + j * gs;
                if (k < nt) {
                    const float4 p = pk[2 * (t0 + k)];
                    ff_inv_log(ff_add(ff{p.x, p.y}, dcx), ff_add(ff{p.z, p.w}, dcy), rho, ln2h, w[j], lg[j], tab);
                }
            }
            for (int kk = P - 1; kk >= 1; kk--) {
                const float4 a = A[kk];
                const cff ak = {{a.x, a.y}, {a.z, a.w}};
#pragma unroll
                for (int j = 0; j < MAXPL; j++)
                    if (gl + j * gs < nt) h[j] = cff_fma(h[j], w[j], ak);
            }
#pragma unroll
            for (int j = 0; j < MAXPL; j++)
                if (gl + j * gs < nt) {
                    const ff re = ff_dot2(h[j].re, w[j].re, h[j].im, w[j].im, ff_mul(ff{a0.x, a0.y}, lg[j]));
                    ar[j] = ff_add(ar[j], re);
                }
            // leaves of more than MAXPL gs points: the rest one at a time, added directly
            for (int32_t k = gl + MAXPL * gs; k < nt; k += gs) {
                const float4 p = pk[2 * (t0 + k)];
                cff w1, h1 = {{0.f, 0.f}, {0.f, 0.f}};
                ff lg1;
                ff_inv_log(ff_add(ff{p.x, p.y}, dcx), ff_add(ff{p.z, p.w}, dcy), rho, ln2h, w1, lg1, tab);
                for (int kk = P - 1; kk >= 1; kk--) {
                    const float4 a = A[kk];
                    h1 = cff_fma(h1, w1, cff{{a.x, a.y}, {a.z, a.w}});
                }
                const ff re = ff_dot2(h1.re, w1.re, h1.im, w1.im, ff_mul(ff{a0.x, a0.y}, lg1));
                atomicAdd(acc + t0 + k, (double)re.h + (double)re.l);
            }
        }
        flush();
    }
}

// Split-mode P2L: the walk of k_p2l (a warp per target leaf, the points of its P2L sources 32 at
// a time, a lane per point) in float-float: u = rho_t / dz from the point's float-float offset
// plus the binary64 centre difference c_s - c_g, the terms q log|dz| and q u^l through shared
// memory (a float-float complex value per coefficient), the column sums in float-float; the leaf's
// sums are added to its binary64 local expansion (b~_0 += sum q log|dz|, b~_l -= sum q u^l / l).
// schedule: the leaves, WPB per block (the P2M schedule)
__global__ void k_p2l_ff(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs, int P, int PS,
                         const int32_t* __restrict__ lb, const float4* __restrict__ pk,
                         const double* __restrict__ cen, const double* __restrict__ rad, XLists xl,
                         cx<double>* __restrict__ Le)
{
    extern __shared__ unsigned char smem[];
    __shared__ float tab[3][129];  // the logarithm's table (see ff_log2)
    for (int i = threadIdx.x; i < 3 * 129; i += blockDim.x) (&tab[0][0])[i] = (&c_lg2t[0][0])[i];
    __syncthreads();
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const int L = S.L;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    if (L < 1) return;
    lb += S.lb0;
    pk += 2 * S.p0;
    cen += 2 * S.b0;
    rad += S.b0;
    Le += S.b0 * PS;
    const int32_t* xoff = xl.xoff + S.o0;
    const int32_t* xidx = xl.xidx + LIs[z.i].s0;
    const int64_t base = level_base(L);
    const ff ln2h = ff_split(0.34657359027997264);  // ln(2) / 2
    cff* Sm = (cff*)smem + (size_t)w * 33 * P;
    for (int64_t b = (int64_t)z.rank * wpb + w; b < level_size(L); b += (int64_t)z.nb * wpb) {
        const int64_t g = base + b;
        const int32_t x0 = xoff[g], x1 = xoff[g + 1];
        if (x0 == x1) continue;
        const ff rho = ff_split(rad[g]);
        cff acc[2] = {{{0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}}};
        ff acc0 = {0.f, 0.f};
        for (int32_t e0 = x0; e0 < x1; e0 += 32) {
            // lane k describes entry e0 + k: its source's first point and count (0 for M2P entries)
            int32_t cnt = 0, first = 0, src = 0;
            if (e0 + lane < x1) {
                const int32_t v = xidx[e0 + lane];
                if (!(v & SWAP_M2P)) {
                    first = lb[v];
                    cnt = lb[v + 1] - first;
                    src = v;
                }
            }
            int32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int32_t excl = incl - cnt, total = __shfl_sync(0xffffffffu, incl, 31);
            for (int32_t f0 = 0; f0 < total; f0 += 32) {
                const int32_t fi = f0 + lane;
                // owner: the last lane k with excl_k <= fi (excl is non-decreasing)
                int k = 0;
#pragma unroll
                for (int st = 16; st; st >>= 1) {
                    const int cand = k + st;
                    const int32_t ec = __shfl_sync(0xffffffffu, excl, cand & 31);
                    if (cand < 32 && ec <= fi) k = cand;
                }
                const int32_t fk = __shfl_sync(0xffffffffu, first, k);
                const int32_t ek = __shfl_sync(0xffffffffu, excl, k);
                const int32_t sk = __shfl_sync(0xffffffffu, src, k);
                cff pw = {{0.f, 0.f}, {0.f, 0.f}}, u = pw;
                ff lg = {0.f, 0.f};
                if (fi < total) {
                    const int64_t ip = fk + (fi - ek);
                    const float4 p = pk[2 * ip], pq = pk[2 * ip + 1];
                    const int64_t sgb = base + sk;
                    const ff dx = ff_add(ff{p.x, p.y}, ff_split(cen[2 * sgb] - cen[2 * g]));
                    const ff dy = ff_add(ff{p.z, p.w}, ff_split(cen[2 * sgb + 1] - cen[2 * g + 1]));
                    ff_inv_log(dx, dy, rho, ln2h, u, lg, tab);
                    const ff q = {pq.x, pq.y};
                    pw.re = q;
                    lg = ff_mul(q, lg);
                }
                Sm[lane] = {lg, {0.f, 0.f}};
                for (int l = 1; l < P; l++) {
                    pw = cff_mul(pw, u);
                    Sm[l * 33 + lane] = pw;
                }
                __syncwarp();
                for (int l = lane, s2 = 0; l < P; l += 32, s2++) {
                    cff sum = Sm[l * 33];
                    for (int j = 1; j < 32; j++) sum = cff_add(sum, Sm[l * 33 + j]);
                    if (l == 0) acc0 = ff_add(acc0, sum.re);
                    else acc[s2] = cff_add(acc[s2], sum);
                }
                __syncwarp();
            }
        }
        cx<double>* B = Le + g * PS;
        for (int l = lane, s2 = 0; l < P; l += 32, s2++) {
            if (l == 0) {
                B[0].re += (double)acc0.h + (double)acc0.l;
            } else {
                const double re = (double)acc[s2].re.h + (double)acc[s2].re.l;
                const double im = (double)acc[s2].im.h + (double)acc[s2].im.l;
                B[l].re -= re / l;
                B[l].im -= im / l;
            }
        }
    }
}

__global__ void k_unpermute(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ perm,
                            const double* __restrict__ acc, double* __restrict__ phi)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    perm += S.p0;
    acc += S.p0;
    phi += S.p0;
    const int64_t n = S.n;
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)z.nb * blockDim.x)
        phi[perm[i]] = acc[i];
}

// The binary64 far field joined with the float-float near field (sums in log2 units), in
// binary64, into input order.
__global__ void k_combine64(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ perm,
                            const double* __restrict__ far, const float* __restrict__ nhi,
                            const float* __restrict__ nlo, double* __restrict__ phi)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    perm += S.p0;
    far += S.p0;
    nhi += S.p0;
    nlo += S.p0;
    phi += S.p0;
    const double scale = 0.34657359027997264;  // ln(2) / 2
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x)
        phi[perm[i]] = far[i] + scale * ((double)nhi[i] + (double)nlo[i]);
}

// binary32 path: phi = far + (ln 2 / 2) * near, combined in binary32 (the mixed path targets
// tolerances >= 1e-7), written in input order.
__global__ void k_combine32(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ perm,
                            const float* __restrict__ far, const float* __restrict__ farlo,
                            const float* __restrict__ nhi, const float* __restrict__ nlo,
                            double* __restrict__ phi)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    perm += S.p0;
    far += S.p0;
    farlo += S.p0;
    nhi += S.p0;
    nlo += S.p0;
    phi += S.p0;
    const int64_t n = S.n;
    const double scale = 0.34657359027997264;  // ln(2) / 2: near-field sums are of log2(r^2)
    // the two float-float sums are joined in binary64 (four additions per point)
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)z.nb * blockDim.x)
        phi[perm[i]] = ((double)far[i] + (double)farlo[i]) + scale * ((double)nhi[i] + (double)nlo[i]);
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


// ---- the complex field of Section 5's first experiment: F_i = sum_{j != i} -q_j / (z_i - z_j) ----
// Far part: minus the derivative of the local expansion, -sum_{l >= 1} l b~_l w^(l-1) / rho with
// w = (z - c) / rho.  Near part: the direct sum along the finest-level strong lists.

__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The binary32 near field works on float-float offsets from the leaf centre (x - c = hi + lo,
// each binary32): a difference of two nearby points then keeps its relative accuracy, so no pair
// needs binary64.  pkf = (x_hi, y_hi, x_lo, y_lo), qf = q, canonical order.
__global__ void k_pack_field32(Sched sc, const Inst* __restrict__ I, const double* __restrict__ q,
                               const int32_t* __restrict__ perm, const double* __restrict__ xs,
                               const double* __restrict__ ys, const float* __restrict__ dxf,
                               const float* __restrict__ dyf, const int32_t* __restrict__ cleaf,
                               const double* __restrict__ cen, float4* __restrict__ pkf, float* __restrict__ qf)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    q += S.p0;
    perm += S.p0;
    xs += S.p0;
    ys += S.p0;
    dxf += S.p0;
    dyf += S.p0;
    cleaf += S.p0;
    pkf += S.p0;
    qf += S.p0;
    cen += 2 * S.b0;
    const int64_t base = level_base(S.L);
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x) {
        const int64_t g = base + cleaf[i];
        const float hx = dxf[i], hy = dyf[i];
        const float lx = __double2float_rn(__dsub_rn(__dsub_rn(xs[i], cen[2 * g]), (double)hx));
        const float ly = __double2float_rn(__dsub_rn(__dsub_rn(ys[i], cen[2 * g + 1]), (double)hy));
        pkf[i] = make_float4(hx, hy, lx, ly);
        qf[i] = (float)q[perm[i]];
    }
}

// far part of the field; a zero-size target leaf (all its points coincide) has no scaled
// derivative: the status word records it (FMM_ERR_DEGENERATE)
template <typename T>
__global__ void k_l2p_field(Sched sc, const Inst* __restrict__ I, int P, int PS, const int32_t* __restrict__ cleaf,
                            const Pk<T>* __restrict__ pk, Geo<T> geo, const cx<T>* __restrict__ Le,
                            T* __restrict__ fre, T* __restrict__ fim, int32_t* status)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const int L = S.L;
    cleaf += S.p0;
    pk += S.p0;
    fre += S.p0;
    fim += S.p0;
    geo = geo.shift(S.b0);
    Le += S.b0 * PS;
    bool degenerate = false;
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x) {
        const int64_t g = level_base(L) + cleaf[i];
        const Pk<T> p = pk[i];
        const T rho = geo.radius(g);
        cx<T> f = {0, 0};
        if (rho > (T)0) {
            const cx<T> w = geo.local(g, p.x, p.y);
            const cx<T>* B = Le + g * PS;
            cx<T> h = {0, 0};
            for (int l = P - 1; l >= 1; l--) h = cfma(h, w, cscale(B[l], (T)l));
            f = cscale(h, (T)-1 / rho);
        } else if (L >= 2) {
            degenerate = true;
        }
        fre[i] = f.re;
        fim[i] = f.im;
    }
    if (__any_sync(0xffffffffu, degenerate) && (threadIdx.x & 31) == 0) atomicOr(status, ST_DEGENERATE);
}

// binary32 near field: the layout of k_p2p_f32 (lane groups on a leaf pair, two targets per lane,
// a run of consecutive leaf pairs per group), with float-float offsets and a binary32 reciprocal;
// coincident points (r = 0, including j = i) contribute nothing.  Accumulators: float-float per
// component, fhr/fhl (real hi, lo) and fir/fil (imaginary hi, lo).
__global__ void __launch_bounds__(256) k_p2p_field_f32(Sched sc, const Inst* __restrict__ I,
                                                       const LInst* __restrict__ LIs,
                                                       const int32_t* __restrict__ soff,
                                                       const int32_t* __restrict__ sidx,
                                                       const int32_t* __restrict__ stgt,
                                                       const int32_t* __restrict__ lb,
                                                       const float4* __restrict__ pkf, const float* __restrict__ qf,
                                                       const float* __restrict__ chi, const float* __restrict__ clo,
                                                       float* __restrict__ fhr, float* __restrict__ flr,
                                                       float* __restrict__ fhi, float* __restrict__ fli)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    const int L = S.L;
    const int64_t scap = TL.scap;
    soff += S.o0;
    sidx += TL.s0;
    stgt += TL.s0;
    lb += S.lb0;
    pkf += S.p0;
    qf += S.p0;
    chi += 2 * S.b0;
    clo += 2 * S.b0;
    fhr += S.p0;
    flr += S.p0;
    fhi += S.p0;
    fli += S.p0;
    const int64_t maxleaf = (int64_t)S.maxleaf;
    if (maxleaf > 64) return;  // left to the general kernel
    int gsl = 1;
    while (2 * gsl < maxleaf) gsl <<= 1;
    const int lane = threadIdx.x & 31, G = 32 / gsl, grp = lane / gsl, li = lane - grp * gsl;
    const int32_t base = (int32_t)level_base(L);
    const int64_t e_begin = min((int64_t)soff[base], scap);
    const int64_t e_end = min((int64_t)soff[base + level_size(L)], scap);
    const int64_t warp = ((int64_t)z.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)z.nb * blockDim.x) >> 5;
    const int64_t wch = (int64_t)G * P2P_GROUP_CH;
    for (int64_t w0 = e_begin + warp * wch; w0 < e_end; w0 += nwarps * wch) {
        const int64_t e0 = w0 + (int64_t)grp * P2P_GROUP_CH;
        const int64_t e1 = min(e0 + P2P_GROUP_CH, e_end);
        int32_t cur = -1, it0 = 0, it1 = 0;
        bool v0 = false, v1 = false;
        float4 ta = make_float4(0.f, 0.f, 0.f, 0.f), tb = ta;
        float ar = 0.f, arl = 0.f, ai = 0.f, ail = 0.f, br = 0.f, brl = 0.f, bi = 0.f, bil = 0.f;
        auto flush = [&]() {
            if (v0) {
                atomicAdd(&fhr[it0], ar);
                atomicAdd(&flr[it0], arl);
                atomicAdd(&fhi[it0], ai);
                atomicAdd(&fli[it0], ail);
            }
            if (v1) {
                atomicAdd(&fhr[it1], br);
                atomicAdd(&flr[it1], brl);
                atomicAdd(&fhi[it1], bi);
                atomicAdd(&fli[it1], bil);
            }
        };
        for (int64_t e = e0; e < e1; e++) {
            const int32_t tl = stgt[e] - base;
            if (tl != cur) {
                flush();
                cur = tl;
                const int32_t t0 = lb[tl], nt = lb[tl + 1] - t0;
                it0 = t0 + li;
                it1 = t0 + li + gsl;
                v0 = li < nt;
                v1 = li + gsl < nt;
                ar = arl = ai = ail = br = brl = bi = bil = 0.f;
                if (v0) ta = pkf[it0];
                if (v1) tb = pkf[it1];
            }
            if (!v0) continue;  // v1 implies v0
            const int32_t sl = sidx[e];
            const int32_t s0 = lb[sl], ns = lb[sl + 1] - s0;
            const int32_t sg = base + sl, tg = base + tl;
            // centre difference c_s - c_t as float-float (two-sum of the high parts)
            float oxh, oxl, oyh, oyl;
            {
                const float a = chi[2 * sg], b = -chi[2 * tg];
                oxh = a + b;
                const float bb = oxh - a;
                oxl = ((a - (oxh - bb)) + (b - bb)) + (clo[2 * sg] - clo[2 * tg]);
                const float c = chi[2 * sg + 1], d = -chi[2 * tg + 1];
                oyh = c + d;
                const float dd = oyh - c;
                oyl = ((c - (oyh - dd)) + (d - dd)) + (clo[2 * sg + 1] - clo[2 * tg + 1]);
            }
            // targets in the source leaf's frame, float-float
            auto to_frame = [](float h, float l, float oh, float ol, float& rh, float& rl) {
                const float b = -oh;
                rh = h + b;
                const float bb = rh - h;
                rl = ((h - (rh - bb)) + (b - bb)) + (l - ol);
            };
            float xah, xal, yah, yal, xbh, xbl, ybh, ybl;
            to_frame(ta.x, ta.z, oxh, oxl, xah, xal);
            to_frame(ta.y, ta.w, oyh, oyl, yah, yal);
            to_frame(tb.x, tb.z, oxh, oxl, xbh, xbl);
            to_frame(tb.y, tb.w, oyh, oyl, ybh, ybl);
            float pra = 0.f, pia = 0.f, prb = 0.f, pib = 0.f;
#pragma unroll 4
            for (int32_t j = 0; j < ns; j++) {
                const float4 sp = pkf[s0 + j];
                const float q = qf[s0 + j];
                const float dxa = (xah - sp.x) + (xal - sp.z), dya = (yah - sp.y) + (yal - sp.w);
                const float dxb = (xbh - sp.x) + (xbl - sp.z), dyb = (ybh - sp.y) + (ybl - sp.w);
                const float ra = dxa * dxa + dya * dya, rb = dxb * dxb + dyb * dyb;
                const float sa = ra > 1e-36f ? q * rcp_fast(ra) : 0.f;
                const float sb = rb > 1e-36f ? q * rcp_fast(rb) : 0.f;
                pra -= sa * dxa;  // -q / dz = -q (dx - i dy) / r^2
                pia += sa * dya;
                prb -= sb * dxb;
                pib += sb * dyb;
            }
            two_sum(ar, arl, pra);
            two_sum(ai, ail, pia);
            if (v1) {
                two_sum(br, brl, prb);
                two_sum(bi, bil, pib);
            }
        }
        flush();
    }
}

// binary64 near field: one warp per leaf pair, one lane per target
__global__ void __launch_bounds__(256) k_p2p_field64(Sched sc, const Inst* __restrict__ I,
                                                     const LInst* __restrict__ LIs,
                                                     const int32_t* __restrict__ soff,
                                                     const int32_t* __restrict__ sidx,
                                                     const int32_t* __restrict__ stgt,
                                                     const int32_t* __restrict__ lb,
                                                     const Pk<double>* __restrict__ pk,
                                                     double* __restrict__ fre, double* __restrict__ fim)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    const int L = S.L;
    const int64_t scap = TL.scap;
    soff += S.o0;
    sidx += TL.s0;
    stgt += TL.s0;
    lb += S.lb0;
    pk += S.p0;
    fre += S.p0;
    fim += S.p0;
    const int lane = threadIdx.x & 31;
    const int64_t base = level_base(L);
    const int64_t e_begin = min((int64_t)soff[base], scap);
    const int64_t e_end = min((int64_t)soff[base + level_size(L)], scap);
    const int64_t warp = ((int64_t)z.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)z.nb * blockDim.x) >> 5;
    for (int64_t e = e_begin + warp; e < e_end; e += nwarps) {
        const int64_t tl = stgt[e] - base, sl = sidx[e];
        const int32_t t0 = lb[tl], nt = lb[tl + 1] - t0, s0 = lb[sl], ns = lb[sl + 1] - s0;
        for (int tc = lane; tc < nt; tc += 32) {
            const Pk<double> p = pk[t0 + tc];
            double sr = 0.0, si = 0.0;
            for (int32_t j = 0; j < ns; j++) {
                const Pk<double> sp = pk[s0 + j];
                const double dx = p.x - sp.x, dy = p.y - sp.y;
                const double r2 = dx * dx + dy * dy;
                if (r2 > 0.0) {
                    const double s_ = sp.q / r2;
                    sr -= s_ * dx;
                    si += s_ * dy;
                }
            }
            atomicAdd(&fre[t0 + tc], sr);
            atomicAdd(&fim[t0 + tc], si);
        }
    }
}

__global__ void k_unpermute_field(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ perm,
                                  const double* __restrict__ ar, const double* __restrict__ ai,
                                  double* __restrict__ fre, double* __restrict__ fim)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    perm += S.p0;
    ar += S.p0;
    ai += S.p0;
    fre += S.p0;
    fim += S.p0;
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x) {
        fre[perm[i]] = ar[i];
        fim[perm[i]] = ai[i];
    }
}

__global__ void k_combine_field32(Sched sc, const Inst* __restrict__ I, const int32_t* __restrict__ perm,
                                  const float* __restrict__ far_r, const float* __restrict__ far_i,
                                  const float* __restrict__ fhr, const float* __restrict__ flr,
                                  const float* __restrict__ fhi, const float* __restrict__ fli,
                                  double* __restrict__ fre, double* __restrict__ fim)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    perm += S.p0;
    far_r += S.p0;
    far_i += S.p0;
    fhr += S.p0;
    flr += S.p0;
    fhi += S.p0;
    fli += S.p0;
    fre += S.p0;
    fim += S.p0;
    for (int64_t i = (int64_t)z.rank * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)z.nb * blockDim.x) {
        fre[perm[i]] = (double)far_r[i] + ((double)fhr[i] + (double)flr[i]);
        fim[perm[i]] = (double)far_i[i] + ((double)fhi[i] + (double)fli[i]);
    }
}

// Direct field at sampled targets (binary64), the reference for the field's error.
__global__ void k_direct_field(const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ q, int64_t n, const int64_t* __restrict__ tgt,
                               double* __restrict__ fre, double* __restrict__ fim)
{
    __shared__ double red[2][32];
    const int64_t i = tgt[blockIdx.x];
    const double xi = x[i], yi = y[i];
    double sr = 0, si = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double dx = xi - x[j], dy = yi - y[j];
        const double r2 = dx * dx + dy * dy;
        if (j != i && r2 > 0.0) {
            sr -= q[j] * dx / r2;
            si += q[j] * dy / r2;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sr;
        red[1][threadIdx.x >> 5] = si;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        sr = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0;
        si = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (threadIdx.x == 0) {
            fre[blockIdx.x] = sr;
            fim[blockIdx.x] = si;
        }
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
    static float bnf[PMAXC * PMAXC];
    for (int i = 0; i < PMAXC * PMAXC; i++) bnf[i] = (float)bn[i / PMAXC][i % PMAXC];
    FMM_CUDA(cudaMemcpyToSymbol(g_binom_f, bnf, sizeof(bnf)));
    FMM_CUDA(cudaMemcpyToSymbol(g_binom_d, bn, sizeof(bn)));
    // the binary32 M2L kernel compiles these coefficients in as immediates: they must agree
    static constexpr std::array<float, PMAXC * PMAXC> compiled =
        mcoef_table(std::make_integer_sequence<int, PMAXC * PMAXC>{});
    for (int i = 0; i < PMAXC * PMAXC; i++)
        if (compiled[i] != mf[i / PMAXC][i % PMAXC])
            return fail(FMM_ERR_STATE, "compiled M2L coefficient (%d, %d) differs from the table", i / PMAXC, i % PMAXC);
    FMM_CUDA(cudaMemcpyToSymbol(c_md, md, sizeof(md)));
    static float lg[3][129];
    for (int j = 0; j <= 128; j++) {
        const double v = log2((double)(128 + j) / 128.0);
        lg[0][j] = (float)v;
        lg[1][j] = (float)(v - (double)lg[0][j]);
        const float F = 1.f + (float)j * (1.f / 128.f);
        lg[2][j] = 1.f / F;  // binary32 division, correctly rounded (as on the device)
    }
    FMM_CUDA(cudaMemcpyToSymbol(c_lg2t, lg, sizeof(lg)));
    g_tab_ready[dev] = true;
    return 0;
}

int alloc_ws(fmm_tree t, int PS, bool f64)
{
    if (f64 && !t->acc && cudaMalloc((void**)&t->acc, 8 * (size_t)t->n) != cudaSuccess)
        return fail(FMM_ERR_OOM, "accumulator");
    if (!f64 && !t->acc32 && cudaMalloc((void**)&t->acc32, 6 * 4 * (size_t)t->n) != cudaSuccess)
        return fail(FMM_ERR_OOM, "accumulator");
    if (!f64 && !t->Lf0lo && cudaMalloc((void**)&t->Lf0lo, 4 * (size_t)t->nbox) != cudaSuccess)
        return fail(FMM_ERR_OOM, "local expansion low parts");
    void** pk = f64 ? &t->pk64 : &t->pk32;
    if (!*pk && cudaMalloc(pk, (f64 ? 32 : 16) * (size_t)t->n) != cudaSuccess)
        return fail(FMM_ERR_OOM, "packed points");
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
    have = PS;
    return 0;
}

template <int PI>
int launch_m2l(fmm_tree t, fmm_lists li, int P, int PS, Geo<float> geo, const cx<float>* Me,
               cx<float>* Le, cudaStream_t s)
{
    if (t->s_m2l.blocks == 0) return 0;
    k_m2l_pairs<float, PI><<<t->s_m2l.blocks, 128, 0, s>>>(t->s_m2l.d, t->dinst, li->dlinst, P, PS, li->woff, li->widx,
                                                li->wrow, geo, Me, Le, t->Lf0lo); note_launch();
    FMM_LAUNCH_CHECK("evaluate: M2L");
    return 0;
}

int dispatch_m2l(fmm_tree t, fmm_lists li, int P, int PS, Geo<float> geo, const cx<float>* Me,
                 cx<float>* Le, cudaStream_t s)
{
    if (P <= 9) return launch_m2l<9>(t, li, P, PS, geo, Me, Le, s);
    if (P <= 13) return launch_m2l<13>(t, li, P, PS, geo, Me, Le, s);
    if (P <= 17) return launch_m2l<17>(t, li, P, PS, geo, Me, Le, s);
    if (P == 18) return launch_m2l<18>(t, li, P, PS, geo, Me, Le, s);
    if (P <= 21) return launch_m2l<21>(t, li, P, PS, geo, Me, Le, s);
    if (P <= 25) return launch_m2l<25>(t, li, P, PS, geo, Me, Le, s);
    if (P <= 31) return launch_m2l<31>(t, li, P, PS, geo, Me, Le, s);
    if (P <= 33) return launch_m2l<33>(t, li, P, PS, geo, Me, Le, s);
    return launch_m2l<41>(t, li, P, PS, geo, Me, Le, s);
}

int dispatch_m2l(fmm_tree t, fmm_lists li, int P, int PS, Geo<double> geo, const cx<double>* Me,
                 cx<double>* Le, cudaStream_t s)
{
    const int NT = 64;
    const size_t sm = (size_t)2 * P * NT * sizeof(cx<double>);
    FMM_CUDA(cudaFuncSetAttribute(k_m2l_pairs_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (t->s_m2l.blocks == 0) return 0;
    k_m2l_pairs_f64<<<t->s_m2l.blocks, NT, sm, s>>>(t->s_m2l.d, t->dinst, li->dlinst, P, PS, li->woff, li->widx,
                                                    li->wrow, geo, Me, Le); note_launch();
    FMM_LAUNCH_CHECK("evaluate: M2L");
    return 0;
}

// Workspace of the general near-field kernel (item counts, their scan), sized by the strong
// capacity; allocated on first use (synchronous).
int p2p_items_ws(fmm_lists li)
{
    if (li->p2p_items) return 0;
    const int64_t m = std::max<int64_t>(li->scap, 1);
    if (cudaMalloc((void**)&li->p2p_items, 4 * (size_t)m) != cudaSuccess ||
        cudaMalloc((void**)&li->p2p_pos, 4 * (size_t)(m + 1)) != cudaSuccess ||
        cudaMalloc((void**)&li->p2p_tmp, 4 * (size_t)scan_tmp_words(m)) != cudaSuccess ||
        cudaMalloc((void**)&li->p2p_zero, 16) != cudaSuccess)  // [0]: 0 (scan base); [2..3]: item total
        return fail(FMM_ERR_OOM, "near-field workspace");
    FMM_CUDA(cudaMemset(li->p2p_zero, 0, 16));
    return 0;
}

// The whole evaluation: the potential into phi, or (fim != nullptr) the complex field into
// phi (real part) and fim (imaginary part).
template <typename T>
int run(fmm_tree t, fmm_lists li, const double* q, int P, double* phi, cudaStream_t s, double* fim = nullptr,
        const StepSync* sync = nullptr, bool near32 = false)
{
    // near32 (binary64 expansions only, the split mode): the near field in float-float (terms
    // and sums, k_p2p_ff), joined to the binary64 far field in binary64
    near32 = near32 && sizeof(T) == 8 && fim == nullptr;
    // with sync the lists are being built on sync->side: wait for them before their first use
    bool lists_waited = false;
    auto wait_lists = [&]() -> int {
        if (sync && !lists_waited) {
            FMM_CUDA(cudaStreamWaitEvent(s, sync->lists_done, 0));
            lists_waited = true;
        }
        return 0;
    };
    const bool f64 = sizeof(T) == 8;
    const bool field = fim != nullptr;
    const int PS = (P + 1) & ~1;
    int rc = alloc_ws(t, PS, f64);
    if (rc) return rc;
    if (near32) {
        if (!t->acc32 && cudaMalloc((void**)&t->acc32, 6 * 4 * (size_t)t->n) != cudaSuccess)
            return fail(FMM_ERR_OOM, "accumulator");
        if (!t->pkff && cudaMalloc(&t->pkff, 32 * (size_t)t->n) != cudaSuccess)
            return fail(FMM_ERR_OOM, "packed points");
        if ((li->mode & FMM_LISTS_EXCHANGE) && t->mff_ps < PS) {  // float-float multipoles for M2P
            cudaFree(t->mff);
            t->mff = nullptr;
            t->mff_ps = 0;
            if (cudaMalloc(&t->mff, 16 * (size_t)t->nbox * PS) != cudaSuccess)
                return fail(FMM_ERR_OOM, "float-float multipoles");
            t->mff_ps = PS;
        }
    }
    if (field) {
        if (f64 && !t->accf && cudaMalloc((void**)&t->accf, 16 * (size_t)t->n) != cudaSuccess)
            return fail(FMM_ERR_OOM, "field accumulator");
        if (!f64 && !t->pkf && (cudaMalloc(&t->pkf, 16 * (size_t)t->n) != cudaSuccess ||
                                cudaMalloc((void**)&t->qf, 4 * (size_t)t->n) != cudaSuccess))
            return fail(FMM_ERR_OOM, "field workspace");
    }
    cx<T>* Me = (cx<T>*)(f64 ? t->Me : t->Mf);
    cx<T>* Le = (cx<T>*)(f64 ? t->Le : t->Lf);
    Pk<T>* pk = (Pk<T>*)(f64 ? t->pk64 : t->pk32);
    const Inst* I = t->dinst;
    const LInst* LI = li->dlinst;
    const int Lmax = t->Lmax;
    const int64_t n = t->n;
    // largest leaf of each instance (leaves are balanced); its largest and smallest value
    int64_t maxleaf = 0, minleaf = INT64_MAX;
    for (int i = 0; i < t->n_inst; i++) {
        const Inst& S = t->hinst[i];
        const int64_t ml = (int64_t)S.maxleaf;
        maxleaf = std::max(maxleaf, ml);
        minleaf = std::min(minleaf, ml);
    }
    const int WPB = 4;
    Geo<T> geo;
    if constexpr (sizeof(T) == 8) geo = Geo<T>{t->centers, t->radii};
    else geo = Geo<T>{t->cen_hi, t->cen_lo, t->rad32};
    float* far32 = t->acc32;        // binary32 path: far field hi, lo; near field hi, lo
    float* farlo = t->acc32 + n;
    float* nhi = t->acc32 + 2 * n;
    float* nlo = t->acc32 + 3 * n;
    const unsigned gpts = (unsigned)t->s_pts.blocks;
    const Sched spts = t->s_pts.d;

    {
        StageScope scope(FMM_STAGE_GATHER, s);
        k_pack<T><<<gpts, 256, 0, s>>>(spts, I, t->perm, q, t->xs, t->ys, t->dxf, t->dyf, pk, t->status);
        note_launch();
        if (near32) {
            k_pack_ff<<<gpts, 256, 0, s>>>(spts, I, t->perm, q, t->xs, t->ys, t->cleaf, t->centers,
                                           (float4*)t->pkff);
            note_launch();
        }
        FMM_CUDA(cudaMemsetAsync(Le, 0, (size_t)t->nbox * PS * sizeof(cx<T>), s));
        if (!f64) FMM_CUDA(cudaMemsetAsync(t->Lf0lo, 0, 4 * (size_t)t->nbox, s));
        FMM_LAUNCH_CHECK("evaluate: gather");
        if (sync) FMM_CUDA(cudaEventRecord(sync->gathered, s));
    }
    if (Lmax >= 1) {
        {
            StageScope scope(FMM_STAGE_P2M, s);
            const size_t sm = (size_t)WPB * 33 * P * sizeof(cx<T>);
            FMM_CUDA(cudaFuncSetAttribute(k_p2m<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_p2m<T><<<t->s_p2m.blocks, 32 * WPB, sm, s>>>(t->s_p2m.d, I, P, PS, t->leaf_begin, pk, geo, Me);
            note_launch();
            FMM_LAUNCH_CHECK("evaluate: P2M");
        }
        // forests: every level of every instance in one persistent launch over the work queue;
        // one instance: a launch per level (measured faster there: 0.11 against 0.20 ms for M2M,
        // 0.13 against 0.32 ms for L2L on 2^20 points)
        const bool queued = t->n_inst > 1;
        const size_t bsm = ((P * P * sizeof(T) + 15) & ~15);
        {
            StageScope scope(FMM_STAGE_M2M, s);
            if (queued) {
                FMM_CUDA(cudaMemsetAsync(qview(t).done_up, 0, (size_t)t->q_counter_bytes, s));
                if ((rc = launch_pass_queue<T, true>(t, P, PS, geo, Me, nullptr, s))) return rc;
            } else {
                for (int l = Lmax - 1; l >= 1; l--) {
                    k_m2m<T><<<t->s_m2m[l].blocks, 32 * WPB, bsm + WPB * P * sizeof(cx<T>), s>>>(
                        t->s_m2m[l].d, I, l, P, PS, geo, Me); note_launch();
                }
                FMM_LAUNCH_CHECK("evaluate: M2M");
            }
        }
        if ((rc = wait_lists())) return rc;
        {
            StageScope scope(FMM_STAGE_M2L, s);
            // tensor cores by default from P = 24 on (on 2^20 clustered points with parent-level
            // lists they take 1.1 ms against 2.3 ms at p = 30, but 0.8 ms against 0.67 ms at
            // p = 20, where the O(P) scaling work around the contraction dominates), unless chosen
            // explicitly or by fmm_autotune
            const bool tc = m2l_tc_supported(P) && (t->m2l_kind == 2 || (t->m2l_kind == 0 && P >= 24));
            if (sizeof(T) == 4 && tc)
                rc = m2l_tc(t, li, P, PS, Me, Le, s);
            else
                rc = dispatch_m2l(t, li, P, PS, geo, Me, Le, s);
            if (rc) return rc;
        }
        {
            StageScope scope(FMM_STAGE_L2L, s);
            if (queued) {
                if ((rc = launch_pass_queue<T, false>(t, P, PS, geo, Le, t->Lf0lo, s))) return rc;
            } else {
                for (int l = 1; l < Lmax; l++) {
                    k_l2l<T><<<t->s_l2l[l].blocks, 32 * WPB, bsm + WPB * P * sizeof(cx<T>), s>>>(
                        t->s_l2l[l].d, I, l, P, PS, geo, Le, t->Lf0lo); note_launch();
                }
                FMM_LAUNCH_CHECK("evaluate: L2L");
            }
        }
    }
    // role exchange (Section 4): P2L into the leaves' local expansions before they are evaluated
    const bool swp = (li->mode & FMM_LISTS_EXCHANGE) != 0 && Lmax >= 1;
    const XLists xl{li->xoff, li->xidx, li->xtgt};
    int gsx = 1;  // lane group of the M2P kernel: the largest leaf, up to a warp
    while (gsx < std::min<int64_t>(maxleaf, 32)) gsx <<= 1;
    if ((rc = wait_lists())) return rc;
    // P2L into the leaves' local expansions (role exchange) before they are evaluated
    auto p2l = [&]() -> int {
        if (!swp) return 0;
        if (near32) {  // split mode: float-float
            const size_t sm = (size_t)WPB * 33 * P * sizeof(cff);
            FMM_CUDA(cudaFuncSetAttribute(k_p2l_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_p2l_ff<<<t->s_p2m.blocks, 32 * WPB, sm, s>>>(t->s_p2m.d, I, LI, P, PS, t->leaf_begin,
                                                           (const float4*)t->pkff, t->centers, t->radii, xl,
                                                           (cx<double>*)Le);
            note_launch();
            FMM_LAUNCH_CHECK("evaluate: P2L");
            return 0;
        }
        const size_t sm = (size_t)WPB * 33 * P * sizeof(cx<T>);
        FMM_CUDA(cudaFuncSetAttribute(k_p2l<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_p2l<T><<<t->s_p2m.blocks, 32 * WPB, sm, s>>>(t->s_p2m.d, I, LI, P, PS, t->leaf_begin, pk, geo, xl, Le,
                                                       t->Lf0lo);
        note_launch();
        FMM_LAUNCH_CHECK("evaluate: P2L");
        return 0;
    };
    if (field) {
        StageScope leaf_scope(FMM_STAGE_LEAF, s);  // P2L, L2P, M2P and the near field
        if ((rc = p2l())) return rc;
        const unsigned gp2p = (unsigned)t->s_p2p.blocks;
        const Sched sp2p = t->s_p2p.d;
        if constexpr (sizeof(T) == 4) {
            float* fr = t->acc32 + 0 * n;
            float* fi = t->acc32 + 1 * n;
            float* hr = t->acc32 + 2 * n;
            float* lr = t->acc32 + 3 * n;
            float* hi = t->acc32 + 4 * n;
            float* lo = t->acc32 + 5 * n;
            FMM_CUDA(cudaMemsetAsync(hr, 0, 4 * 4 * (size_t)n, s));
            k_pack_field32<<<gpts, 256, 0, s>>>(spts, I, q, t->perm, t->xs, t->ys, t->dxf, t->dyf, t->cleaf,
                                                t->centers, (float4*)t->pkf, t->qf); note_launch();
            k_l2p_field<float><<<gpts, 256, 0, s>>>(spts, I, P, PS, t->cleaf, pk, geo, Le, fr, fi, t->status);
            note_launch();
            if (swp) {
                k_m2p<float, true><<<gp2p, 256, 0, s>>>(sp2p, I, LI, P, PS, gsx, t->leaf_begin, pk, geo, xl, Me, hr,
                                                        lr, hi, lo);
                note_launch();
            }
            k_p2p_field_f32<<<gp2p, 256, 0, s>>>(sp2p, I, LI, li->soff, li->sidx, li->stgt, t->leaf_begin,
                                                 (const float4*)t->pkf, t->qf, t->cen_hi, t->cen_lo, hr, lr,
                                                 hi, lo); note_launch();
            k_combine_field32<<<gpts, 256, 0, s>>>(spts, I, t->perm, fr, fi, hr, lr, hi, lo, phi, fim);
            note_launch();
        } else {
            k_l2p_field<double><<<gpts, 256, 0, s>>>(spts, I, P, PS, t->cleaf, pk, geo, Le, t->accf, t->accf + n,
                                                     t->status);
            note_launch();
            if (swp) {
                k_m2p<double, true><<<gp2p, 256, 0, s>>>(sp2p, I, LI, P, PS, gsx, t->leaf_begin, pk, geo, xl, Me,
                                                         t->accf, nullptr, t->accf + n, nullptr);
                note_launch();
            }
            k_p2p_field64<<<gp2p, 256, 0, s>>>(sp2p, I, LI, li->soff, li->sidx, li->stgt, t->leaf_begin,
                                               (const Pk<double>*)pk, t->accf, t->accf + n); note_launch();
            k_unpermute_field<<<gpts, 256, 0, s>>>(spts, I, t->perm, t->accf, t->accf + n, phi, fim);
            note_launch();
        }
        FMM_LAUNCH_CHECK("evaluate: field");
        return 0;
    }
    // potentials.  The near field needs only the packed points and the strong lists, so with sync
    // (binary32 path) it runs on the lists' stream while this one finishes the far field; its
    // accumulators (nhi, nlo) are not touched by the far-field kernels.  The binary64 near field
    // adds into the same accumulator as L2P and stays on this stream, before L2P.
    const bool n32 = !f64 || near32;  // binary32 near field (float-float sums in nhi, nlo)
    const bool overlap = sync != nullptr && n32;
    cudaStream_t ns = overlap ? sync->side : s;
    if (overlap) FMM_CUDA(cudaStreamWaitEvent(ns, sync->gathered, 0));
    if (near32) FMM_CUDA(cudaMemsetAsync(t->acc, 0, 8 * (size_t)n, s));  // the far field's accumulator
    {
        StageScope near_scope(FMM_STAGE_NEAR, ns);
        if (!n32) FMM_CUDA(cudaMemsetAsync(t->acc, 0, 8 * (size_t)n, ns));
        else FMM_CUDA(cudaMemsetAsync(nhi, 0, 2 * 4 * (size_t)n, ns));
        const unsigned gp2p = (unsigned)t->s_p2p.blocks;
        const Sched sp2p = t->s_p2p.d;
        const Pk<float>* pk32 = (const Pk<float>*)t->pk32;
        // instances whose leaves hold at most SMALL_LEAF points take the leaf-pair kernel, the
        // others (if any) the general one; each kernel skips the instances of the other (the
        // float-float near field takes the general kernel's work items for every instance)
        const int small_leaf = near32 ? 0 : n32 ? 64 : 32;
        if (!near32 && minleaf <= small_leaf) {
            if (n32) {
                if (t->tune_p2p_nt == 4)
                    k_p2p_f32<4><<<gp2p, 256, 0, ns>>>(sp2p, I, LI, li->soff, li->sidx, li->stgt, t->leaf_begin,
                                                       pk32, t->xs, t->ys, t->cen_hi, t->cen_lo, t->rad32, nhi, nlo);
                else
                    k_p2p_f32<2><<<gp2p, 256, 0, ns>>>(sp2p, I, LI, li->soff, li->sidx, li->stgt, t->leaf_begin,
                                                       pk32, t->xs, t->ys, t->cen_hi, t->cen_lo, t->rad32, nhi, nlo);
            } else {
                int gs = 1;
                while (gs < std::min<int64_t>(maxleaf, 32)) gs <<= 1;
                k_p2p_small<T><<<gp2p, 256, 0, ns>>>(sp2p, I, LI, gs, li->soff, li->sidx, li->stgt,
                                                     t->leaf_begin, pk, t->xs, t->ys, t->cen_hi,
                                                     t->cen_lo, t->rad32, t->acc, nhi, nlo);
            }
            note_launch();
        }
        if (maxleaf > small_leaf) {
            rc = p2p_items_ws(li);
            if (rc) return rc;
            unsigned long long* total = (unsigned long long*)(li->p2p_zero + 2);
            FMM_CUDA(cudaMemsetAsync(total, 0, 8, ns));
            k_p2p_items<<<gp2p, 256, 0, ns>>>(sp2p, I, LI, small_leaf, li->soff, li->sidx, li->stgt, t->leaf_begin,
                                              li->p2p_items, total); note_launch();
            rc = scan_with_base(li->p2p_items, li->scap, li->p2p_zero, li->p2p_pos, li->p2p_tmp, ns);
            if (rc) return rc;
            if (near32)
                k_p2p_ff<<<gp2p, 256, 0, ns>>>(sp2p, I, LI, li->soff, li->sidx, li->stgt, t->leaf_begin, li->p2p_pos,
                                               total, t->status, (const float4*)t->pkff, t->centers, nhi, nlo);
            else if (n32)
                k_p2p_large<float><<<gp2p, 256, 0, ns>>>(sp2p, I, LI, small_leaf, li->soff, li->sidx, li->stgt,
                                                         t->leaf_begin, li->p2p_pos, total, t->status, pk32, t->xs,
                                                         t->ys, t->cen_hi, t->cen_lo, t->rad32, t->acc, nhi, nlo);
            else
                k_p2p_large<T><<<gp2p, 256, 0, ns>>>(sp2p, I, LI, small_leaf, li->soff, li->sidx, li->stgt,
                                                     t->leaf_begin, li->p2p_pos, total, t->status, pk, t->xs, t->ys,
                                                     t->cen_hi, t->cen_lo, t->rad32, t->acc, nhi, nlo);
            note_launch();
        }
        FMM_LAUNCH_CHECK("evaluate: near field");
    }
    if (overlap) FMM_CUDA(cudaEventRecord(sync->near_done, ns));
    {
        // role exchange: P2L into the leaves' local expansions, M2P into the far accumulator
        // (the binary32 one is cleared first, and L2P then adds to it)
        if (swp) {
            StageScope x_scope(FMM_STAGE_EXCHANGE, s);
            if ((rc = p2l())) return rc;
            if (near32) {  // split mode: float-float, from a float-float copy of the multipoles
                const int64_t count = t->nbox * PS;
                k_coeffs_ff<<<(unsigned)std::min<int64_t>((count + 255) / 256, 152 * 16), 256, 0, s>>>(
                    (const double2*)Me, count, (float4*)t->mff);
                note_launch();
                k_m2p_ff<<<(unsigned)t->s_p2p.blocks, 256, 0, s>>>(t->s_p2p.d, I, LI, P, PS, gsx, t->leaf_begin,
                                                                   (const float4*)t->pkff, t->centers, t->radii,
                                                                   xl, (const float4*)t->mff, t->acc);
            } else {
                if (!f64) FMM_CUDA(cudaMemsetAsync(far32, 0, 2 * 4 * (size_t)n, s));  // far32, farlo
                k_m2p<T, false><<<(unsigned)t->s_p2p.blocks, 256, 0, s>>>(t->s_p2p.d, I, LI, P, PS, gsx,
                                                                         t->leaf_begin, pk, geo, xl, Me,
                                                                         f64 ? (T*)t->acc : (T*)far32, farlo,
                                                                         nullptr, nullptr);
            }
            note_launch();
        }
        StageScope leaf_scope(FMM_STAGE_LEAF, s);  // L2P, far and near joined
        k_l2p<T><<<gpts, 256, 0, s>>>(spts, I, P, PS, t->cleaf, pk, geo, Le, t->Lf0lo,
                                      f64 ? (T*)t->acc : (T*)far32, farlo, swp);
        note_launch();
        if (overlap) FMM_CUDA(cudaStreamWaitEvent(s, sync->near_done, 0));
        if (near32)
            k_combine64<<<gpts, 256, 0, s>>>(spts, I, t->perm, t->acc, nhi, nlo, phi);
        else if (f64)
            k_unpermute<<<gpts, 256, 0, s>>>(spts, I, t->perm, t->acc, phi);
        else
            k_combine32<<<gpts, 256, 0, s>>>(spts, I, t->perm, far32, farlo, nhi, nlo, phi);
        note_launch();
        FMM_LAUNCH_CHECK("evaluate: leaf evaluation");
    }
    return 0;
}

}  // namespace

int evaluate(fmm_tree t, fmm_lists li, const double* q, const fmm_params& prm, double* phi,
             cudaStream_t s, const StepSync* sync)
{
    int rc = ensure_tables();
    if (rc) return rc;
    const int P = prm.p + 1;
    // the mixed mode below the binary32 floor takes the split precision: binary64 expansions (the
    // far field needs them: binary32 coefficients carry about 1e-7 of the potential) and the
    // float-float near field, which on GB300 costs a fraction of a binary64 one (slow binary64
    // units) at binary64 accuracy
    const bool split = prm.mode == FMM_MODE_SPLIT ||
                       (prm.mode == FMM_MODE_MIXED && prm.tol > 0.0 && prm.tol < MIXED_TOL_FLOOR);
    if (split) return run<double>(t, li, q, P, phi, s, nullptr, sync, true);
    if (prm.mode == FMM_MODE_FP64) return run<double>(t, li, q, P, phi, s, nullptr, sync);
    return run<float>(t, li, q, P, phi, s, nullptr, sync);
}

// Launch-shape tuner: times complete evaluations (CUDA events on the caller's stream, best of
// three after one warm-up) for a ladder of grid sizes of the two dominant kernels, the M2L pair
// kernel first and then the near-field kernel, and keeps the fastest of each.
int autotune(fmm_tree t, fmm_lists li, const double* q, const fmm_params& prm, double* phi,
             cudaStream_t s, int* m2l_blocks, int* p2p_blocks)
{
    cudaEvent_t e0, e1;
    FMM_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(FMM_ERR_CUDA, "cudaEventCreate");
    }
    auto time_one = [&](float& best) -> int {
        best = 1e30f;
        for (int r = 0; r < 4; r++) {
            FMM_CUDA(cudaEventRecord(e0, s));
            int rc = evaluate(t, li, q, prm, phi, s);
            if (rc) return rc;
            FMM_CUDA(cudaEventRecord(e1, s));
            FMM_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            FMM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) best = std::min(best, ms);
        }
        return 0;
    };
    // Launch shapes: the M2L kernel (SIMT or tensor cores) with its total block count and, for the
    // tensor-core kernel, the consecutive weak entries per row (its tile-to-pair shape); then the
    // near field's total block count.  Each candidate is timed on whole evaluations.
    const int ladder[] = {152, 152 * 2, 152 * 4, 152 * 8, 152 * 16, 152 * 32, 152 * 64};
    const int ladder_tc[] = {152, 152 * 2, 152 * 3, 152 * 4, 152 * 6};
    const int chunks_tc[] = {8, 16, 32};
    int rc = 0;
    const int kind0 = t->m2l_kind, chunk0 = t->tune_m2l_chunk, stages0 = t->tune_m2l_stages;
    const int nt0 = t->tune_p2p_nt;
    t->tune_m2l_blocks = t->tune_p2p_blocks = 0;
    if ((rc = sched_tuned(t))) return rc;
    const bool try_tc = prm.mode == FMM_MODE_MIXED && !(prm.tol > 0.0 && prm.tol < MIXED_TOL_FLOOR) &&
                        m2l_tc_supported(prm.p + 1);
    {
        int best_kind = kind0, best_blocks = 0, best_chunk = chunk0, best_stages = stages0;
        float best_ms = 1e30f;
        auto consider = [&](int kind, int v, int ch, int st) -> int {
            t->m2l_kind = kind;
            t->tune_m2l_blocks = v;
            t->tune_m2l_chunk = ch;
            t->tune_m2l_stages = st;
            int r = sched_tuned(t);
            float ms = 0.f;
            if (!r) r = time_one(ms);
            if (!r && ms < best_ms) {
                best_ms = ms;
                best_kind = kind;
                best_blocks = v;
                best_chunk = ch;
                best_stages = st;
            }
            return r;
        };
        for (int v : ladder)
            if (!rc) rc = consider(try_tc ? 1 : kind0, v, chunk0, stages0);
        if (try_tc)
            for (int v : ladder_tc)
                for (int ch : chunks_tc)
                    for (int st = 1; st <= 2 && !rc; st++) rc = consider(2, v, ch, st);
        t->m2l_kind = best_kind;
        t->tune_m2l_blocks = best_blocks;
        t->tune_m2l_chunk = best_chunk;
        t->tune_m2l_stages = best_stages;
    }
    if (!rc) {
        // near field: block count and, for the binary32 leaf-pair kernel, targets per lane
        const bool try_nt = prm.mode == FMM_MODE_MIXED && !(prm.tol > 0.0 && prm.tol < MIXED_TOL_FLOOR);
        int best_v = 0, best_nt = nt0;
        float best_ms = 1e30f;
        for (int nt : {2, 4}) {
            if (!try_nt && nt != 2) break;
            t->tune_p2p_nt = try_nt ? nt : nt0;
            for (int v : ladder) {
                t->tune_p2p_blocks = v;
                if ((rc = sched_tuned(t))) break;
                float ms = 0.f;
                if ((rc = time_one(ms))) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_v = v;
                    best_nt = t->tune_p2p_nt;
                }
            }
            if (rc) break;
        }
        t->tune_p2p_blocks = best_v;
        t->tune_p2p_nt = best_nt;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) rc = sched_tuned(t);
    if (rc) {
        t->tune_m2l_blocks = t->tune_p2p_blocks = 0;
        t->tune_m2l_chunk = chunk0;
        t->tune_m2l_stages = stages0;
        t->tune_p2p_nt = nt0;
        t->m2l_kind = kind0;
        sched_tuned(t);
        return rc;
    }
    if (m2l_blocks) *m2l_blocks = t->tune_m2l_blocks;
    if (p2p_blocks) *p2p_blocks = t->tune_p2p_blocks;
    return 0;
}

int queues_make(fmm_tree t)
{
    const int ni = t->n_inst;
    std::vector<QItem> up, dn;
    std::vector<int32_t> nup((size_t)ni * QLEVELS, 0), ndn((size_t)ni * QLEVELS, 0);
    for (int l = t->Lmax - 1; l >= 1; l--)
        for (int i = 0; i < ni; i++)
            if (l < t->hinst[i].L)
                for (int64_t b0 = 0; b0 < level_size(l); b0 += QBOX) {
                    up.push_back(QItem{i, l, (int32_t)b0, (int32_t)std::min<int64_t>(QBOX, level_size(l) - b0)});
                    nup[(size_t)i * QLEVELS + l]++;
                }
    for (int l = 1; l < t->Lmax; l++)
        for (int i = 0; i < ni; i++)
            if (l < t->hinst[i].L)
                for (int64_t b0 = 0; b0 < level_size(l); b0 += QBOX) {
                    dn.push_back(QItem{i, l, (int32_t)b0, (int32_t)std::min<int64_t>(QBOX, level_size(l) - b0)});
                    ndn[(size_t)i * QLEVELS + l]++;
                }
    t->nq_up = (int32_t)up.size();
    t->nq_dn = (int32_t)dn.size();
    t->q_counter_bytes = (int64_t)(2 * (size_t)ni * QLEVELS + 2) * sizeof(uint32_t);
    const size_t bytes = (up.size() + dn.size()) * sizeof(QItem) + 2 * (size_t)ni * QLEVELS * sizeof(int32_t) +
                         (size_t)t->q_counter_bytes;
    if (cudaMalloc(&t->qmem, bytes) != cudaSuccess) return fail(FMM_ERR_OOM, "work queues");
    const QView v = qview(t);
    if (!up.empty()) FMM_CUDA(cudaMemcpy(v.up, up.data(), up.size() * sizeof(QItem), cudaMemcpyHostToDevice));
    if (!dn.empty()) FMM_CUDA(cudaMemcpy(v.dn, dn.data(), dn.size() * sizeof(QItem), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemcpy(v.need_up, nup.data(), nup.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemcpy(v.need_dn, ndn.data(), ndn.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemset(v.done_up, 0, (size_t)t->q_counter_bytes));
    return 0;
}

// The queued upward pass with a dependency that never completes: instance 0's item count of its
// deepest M2M level is raised by one in a copy of the needs, so the items of the level above wait
// for an item that is not in the queue.  Each wait gives up after `limit` tries; the pass runs on
// scratch coefficients (p = 3) and a scratch status word, which is read back.
int queue_timeout_selftest(fmm_tree t, int64_t limit, cudaStream_t s)
{
    const Inst& S = t->hinst[0];
    if (S.L < 3) return fail(FMM_ERR_ARG, "the self-test needs an instance of at least 3 levels");
    int rc = ensure_tables();
    if (rc) return rc;
    const int P = 4, PS = 4;
    const QView v = qview(t);
    const size_t nneed = (size_t)t->n_inst * QLEVELS;
    std::vector<int32_t> need(nneed);
    cx<double>* E = nullptr;
    int32_t* dneed = nullptr;
    int32_t* st = nullptr;
    auto cleanup = [&]() {
        cudaFree(E);
        cudaFree(dneed);
        cudaFree(st);
    };
    if (cudaMalloc((void**)&E, sizeof(cx<double>) * PS * (size_t)t->nbox) != cudaSuccess ||
        cudaMalloc((void**)&dneed, 4 * nneed) != cudaSuccess || cudaMalloc((void**)&st, 4) != cudaSuccess) {
        cleanup();
        return fail(FMM_ERR_OOM, "self-test scratch");
    }
    int32_t h = 0;
    rc = [&]() -> int {
        FMM_CUDA(cudaStreamSynchronize(s));
        FMM_CUDA(cudaMemcpy(need.data(), v.need_up, 4 * nneed, cudaMemcpyDeviceToHost));
        need[(size_t)0 * QLEVELS + (S.L - 1)] += 1;  // a producer that is not in the queue
        FMM_CUDA(cudaMemcpy(dneed, need.data(), 4 * nneed, cudaMemcpyHostToDevice));
        FMM_CUDA(cudaMemsetAsync(E, 0, sizeof(cx<double>) * PS * (size_t)t->nbox, s));
        FMM_CUDA(cudaMemsetAsync(st, 0, 4, s));
        FMM_CUDA(cudaMemsetAsync(v.done_up, 0, (size_t)t->q_counter_bytes, s));
        int r = launch_pass_queue<double, true>(t, P, PS, Geo<double>{t->centers, t->radii}, E, nullptr, s, dneed,
                                                st, limit);
        if (r) return r;
        FMM_CUDA(cudaStreamSynchronize(s));
        FMM_CUDA(cudaMemcpy(&h, st, 4, cudaMemcpyDeviceToHost));
        return 0;
    }();
    cleanup();
    if (rc) return rc;
    return (h & ST_TIMEOUT) ? fail(FMM_ERR_TIMEOUT, "a queued item gave up waiting after %lld tries, as it should",
                                   (long long)limit)
                            : FMM_OK;
}

int evaluate_field(fmm_tree t, fmm_lists li, const double* q, const fmm_params& prm, double* fre,
                   double* fim, cudaStream_t s)
{
    int rc = ensure_tables();
    if (rc) return rc;
    const int P = prm.p + 1;
    int64_t maxleaf = 0;
    for (int i = 0; i < t->n_inst; i++) {
        const Inst& S = t->hinst[i];
        maxleaf = std::max<int64_t>(maxleaf, (int64_t)S.maxleaf);
    }
    // the binary32 near-field kernel holds up to 64 targets per leaf; larger leaves, tolerances
    // below the binary32 floor and binary64 mode take the binary64 path
    const bool f64 = prm.mode != FMM_MODE_MIXED || (prm.tol > 0.0 && prm.tol < MIXED_TOL_FLOOR) || maxleaf > 64;
    if (f64) return run<double>(t, li, q, P, fre, s, fim);
    return run<float>(t, li, q, P, fre, s, fim);
}

int direct_field(const double* x, const double* y, const double* q, int64_t n, const int64_t* tgt,
                 int64_t m, double* fre, double* fim, cudaStream_t s)
{
    if (m <= 0) return 0;
    for (int64_t off = 0; off < m; off += 65535) {
        const int64_t c = std::min<int64_t>(65535, m - off);
        k_direct_field<<<(unsigned)c, 256, 0, s>>>(x, y, q, n, tgt + off, fre + off, fim + off); note_launch();
    }
    FMM_LAUNCH_CHECK("direct field");
    return 0;
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
