// The parameter selector's network: a multilayer perceptron 64 -> 128 -> 128 -> 225 with ReLU
// hidden layers and a softmax over the 225 (levels, p) classes, trained with softmax
// cross-entropy and Adam.  The paper has no counterpart: it fixes the parameters by the rules at
// the end of Section 4 (p ~ log TOL / log theta from the analysis of Section 3, about 20 points
// per leaf); the network learns the fastest (levels, p) that meets a tolerance from runs of the
// method itself.
//
// Everything runs in binary32 on the GPU: one tiled matrix-product kernel with optional
// transposes and a fused epilogue (bias, ReLU, or the ReLU derivative mask), a row-wise softmax
// with the cross-entropy gradient, a column-sum for the bias gradients and the Adam update.  The
// matrices are tiny (batch x 225 at most), so the kernels use the SIMT units.
//
// Parameter layout (one flat binary32 array, row-major): W1[128][64], b1[128], W2[128][128],
// b2[128], W3[225][128], b3[225] -- 53,857 values.
#include <algorithm>
#include <new>

#include "common.cuh"

struct fmm_mlp_s {
    int dev = 0;
    int bmax = 0;
    float* params = nullptr;  // [FMM_MLP_PARAMS]
    float* grads = nullptr;
    float* m = nullptr;       // Adam moments
    float* v = nullptr;
    float* h1 = nullptr;      // [bmax][128]
    float* h2 = nullptr;      // [bmax][128]
    float* z = nullptr;       // [bmax][225] logits, then probabilities
    float* dz = nullptr;      // [bmax][225]
    float* dh2 = nullptr;     // [bmax][128]
    float* dh1 = nullptr;     // [bmax][128]
    float* loss = nullptr;    // [bmax] per-sample loss, [1] mean after the reduction
    float* lossm = nullptr;
    int64_t step = 0;
};

namespace fmm {
namespace {

constexpr int D0 = FMM_MLP_IN, D1 = FMM_MLP_HIDDEN, D2 = FMM_MLP_HIDDEN, D3 = FMM_MLP_OUT;
constexpr int64_t OW1 = 0, OB1 = OW1 + (int64_t)D1 * D0, OW2 = OB1 + D1, OB2 = OW2 + (int64_t)D2 * D1,
                  OW3 = OB2 + D2, OB3 = OW3 + (int64_t)D3 * D2, NPAR = OB3 + D3;
static_assert(NPAR == FMM_MLP_PARAMS, "parameter count");

enum Epi { EPI_NONE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_MASK = 3 };

constexpr int GT = 32;  // output tile edge; 256 threads compute 2 x 2 outputs each

// C[M][N] = sum_k A'(i,k) B'(k,j), with A'(i,k) = TA ? A[k*lda+i] : A[i*lda+k] and
// B'(k,j) = TB ? B[j*ldb+k] : B[k*ldb+j]; epilogue: + bias[j] (and ReLU), or * (mask[i][j] > 0).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, float* __restrict__ C,
                                              int ldc, int epi, const float* __restrict__ bias,
                                              const float* __restrict__ mask)
{
    __shared__ float As[GT][GT + 1];  // As[k][i]
    __shared__ float Bs[GT][GT + 1];  // Bs[k][j]
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k0 = 0; k0 < K; k0 += GT) {
        for (int e = threadIdx.x; e < GT * GT; e += 256) {
            const int r = e / GT, c = e % GT;
            // A tile: element (i = i0 + ri, k = k0 + rk)
            {
                const int ri = TA ? c : r, rk = TA ? r : c;
                const int i = i0 + ri, k = k0 + rk;
                As[rk][ri] = (i < M && k < K) ? (TA ? A[(int64_t)k * lda + i] : A[(int64_t)i * lda + k]) : 0.f;
            }
            {
                const int rj = TB ? r : c, rk = TB ? c : r;
                const int j = j0 + rj, k = k0 + rk;
                Bs[rk][rj] = (j < N && k < K) ? (TB ? B[(int64_t)j * ldb + k] : B[(int64_t)k * ldb + j]) : 0.f;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < GT; k++) {
            const float a0 = As[k][ty], a1 = As[k][ty + 16];
            const float b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
            acc[0][0] = fmaf(a0, b0, acc[0][0]);
            acc[0][1] = fmaf(a0, b1, acc[0][1]);
            acc[1][0] = fmaf(a1, b0, acc[1][0]);
            acc[1][1] = fmaf(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int w = 0; w < 2; w++) {
            const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * w;
            if (i >= M || j >= N) continue;
            float c = acc[u][w];
            if (epi == EPI_BIAS_RELU) c = fmaxf(c + bias[j], 0.f);
            else if (epi == EPI_BIAS) c += bias[j];
            else if (epi == EPI_MASK) c = mask[(int64_t)i * ldc + j] > 0.f ? c : 0.f;
            C[(int64_t)i * ldc + j] = c;
        }
}

template <bool TA, bool TB>
void gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc, int epi,
          const float* bias, const float* mask, cudaStream_t s)
{
    const dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    k_gemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, epi, bias, mask);
    note_launch();
}

// Row-wise softmax of the logits (in place) and, with labels, the per-sample cross-entropy and
// its gradient (p - onehot) / B.  One warp per row.
__global__ void k_softmax_xent(int B, float* __restrict__ z, const int32_t* __restrict__ label,
                               float* __restrict__ dz, float* __restrict__ loss)
{
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= B) return;
    float* zr = z + (int64_t)row * D3;
    float mx = -3.0e38f;
    for (int j = lane; j < D3; j += 32) mx = fmaxf(mx, zr[j]);
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float sum = 0.f;
    for (int j = lane; j < D3; j += 32) sum += expf(zr[j] - mx);
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const float lse = mx + logf(sum);
    const int y = label ? label[row] : -1;
    if (label && lane == 0 && (y < 0 || y >= D3)) loss[row] = __int_as_float(0x7fc00000);  // NaN: bad label
    for (int j = lane; j < D3; j += 32) {
        const float lz = zr[j] - lse;
        const float p = expf(lz);
        if (label) {
            dz[(int64_t)row * D3 + j] = (p - (j == y ? 1.f : 0.f)) / (float)B;
            if (j == y) loss[row] = -lz;
        }
        zr[j] = p;
    }
}

// out[j] = scale * sum_i in[i][j] (bias gradients).
__global__ void k_colsum(int B, int N, const float* __restrict__ in, float* __restrict__ out, float scale)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int i = 0; i < B; i++) s += in[(int64_t)i * N + j];
    out[j] = s * scale;
}

// Adam (Kingma and Ba, 2015) with bias correction.
__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Masked arg-max over the classes (levels = 4 + c / 25, p = 8 + c % 25): classes whose levels
// exceed log4(N) (N from feature 60 = log10 N) are left out.  One warp per sample.
__global__ void k_select(int B, const float* __restrict__ prob, const float* __restrict__ feat,
                         int32_t* __restrict__ out)
{
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= B) return;
    const double n = pow(10.0, (double)feat[(int64_t)row * D0 + FMM_FEAT_LOG10N]) * (1.0 + 1e-6);
    int lmax = FMM_SEL_LMIN;
    while (lmax + 1 <= FMM_SEL_LMAX && ldexp(1.0, 2 * (lmax + 1)) <= n) lmax++;
    // the window the training labels come from: Lc - 2 .. Lc + 1 around Lc = round(log4(N / 32))
    // (half up), i.e. Lc = floor((b - 4) / 2) with b = floor(log2 N)
    int b = 0;
    while (b < 62 && ldexp(1.0, b + 1) <= n) b++;
    const int lc = b >= 4 ? (b - 4) / 2 : -((5 - b) / 2);
    const int wlo = max(FMM_SEL_LMIN, lc - 2), whi = min(lmax, lc + 1);
    const int lo = wlo <= whi ? wlo : FMM_SEL_LMIN, hi = wlo <= whi ? whi : lmax;
    float best = -1.f;
    int bi = 0;
    for (int c = lane; c < D3; c += 32) {
        const int L = FMM_SEL_LMIN + c / FMM_SEL_NP;
        const float pc = prob[(int64_t)row * D3 + c];
        if (L >= lo && L <= hi && pc > best) {
            best = pc;
            bi = c;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    if (lane == 0) {
        out[2 * row] = FMM_SEL_LMIN + bi / FMM_SEL_NP;
        out[2 * row + 1] = FMM_SEL_PMIN + bi % FMM_SEL_NP;
    }
}

void forward(fmm_mlp m, const float* X, int B, cudaStream_t s)
{
    const float* P = m->params;
    gemm<false, true>(B, D1, D0, X, D0, P + OW1, D0, m->h1, D1, EPI_BIAS_RELU, P + OB1, nullptr, s);
    gemm<false, true>(B, D2, D1, m->h1, D1, P + OW2, D1, m->h2, D2, EPI_BIAS_RELU, P + OB2, nullptr, s);
    gemm<false, true>(B, D3, D2, m->h2, D2, P + OW3, D2, m->z, D3, EPI_BIAS, P + OB3, nullptr, s);
}

// Forward, softmax cross-entropy and backward: gradients into m->grads, mean loss into m->lossm.
int grads(fmm_mlp m, const float* X, const int32_t* label, int B, cudaStream_t s)
{
    forward(m, X, B, s);
    k_softmax_xent<<<(B + 7) / 8, 256, 0, s>>>(B, m->z, label, m->dz, m->loss); note_launch();
    float* G = m->grads;
    const float* P = m->params;
    // layer 3: dW3 = dZ^T H2, db3 = sum dZ, dH2 = (dZ W3) * (H2 > 0)
    gemm<true, false>(D3, D2, B, m->dz, D3, m->h2, D2, G + OW3, D2, EPI_NONE, nullptr, nullptr, s);
    k_colsum<<<(D3 + 127) / 128, 128, 0, s>>>(B, D3, m->dz, G + OB3, 1.f); note_launch();
    gemm<false, false>(B, D2, D3, m->dz, D3, P + OW3, D2, m->dh2, D2, EPI_MASK, nullptr, m->h2, s);
    // layer 2
    gemm<true, false>(D2, D1, B, m->dh2, D2, m->h1, D1, G + OW2, D1, EPI_NONE, nullptr, nullptr, s);
    k_colsum<<<(D2 + 127) / 128, 128, 0, s>>>(B, D2, m->dh2, G + OB2, 1.f); note_launch();
    gemm<false, false>(B, D1, D2, m->dh2, D2, P + OW2, D1, m->dh1, D1, EPI_MASK, nullptr, m->h1, s);
    // layer 1
    gemm<true, false>(D1, D0, B, m->dh1, D1, X, D0, G + OW1, D0, EPI_NONE, nullptr, nullptr, s);
    k_colsum<<<(D1 + 127) / 128, 128, 0, s>>>(B, D1, m->dh1, G + OB1, 1.f); note_launch();
    FMM_LAUNCH_CHECK("mlp: gradients");
    return 0;
}

// mean of the per-sample losses (one block)
__global__ void k_mean(int B, const float* __restrict__ in, float* __restrict__ out)
{
    __shared__ float part[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < B; i += blockDim.x) s += in[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = part[0] / (float)B;
}

int grads_and_loss(fmm_mlp m, const float* X, const int32_t* label, int B, cudaStream_t s)
{
    int rc = grads(m, X, label, B, s);
    if (rc) return rc;
    k_mean<<<1, 256, 0, s>>>(B, m->loss, m->lossm); note_launch();
    FMM_LAUNCH_CHECK("mlp: loss");
    return 0;
}

struct Guard {
    int prev = -1;
    bool ok = true;
    explicit Guard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~Guard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void free_mlp(fmm_mlp m)
{
    void* ptrs[] = {m->params, m->grads, m->m, m->v, m->h1, m->h2, m->z, m->dz, m->dh2, m->dh1, m->loss, m->lossm};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

int check_batch(fmm_mlp m, int B)
{
    if (!m) return fail(FMM_ERR_ARG, "NULL network");
    if (B < 1 || B > m->bmax) return fail(FMM_ERR_ARG, "batch %d outside [1, %d]", B, m->bmax);
    return 0;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" {

int fmm_mlp_create(int batch_max, fmm_mlp* out)
{
    if (!out) return fail(FMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (batch_max < 1 || batch_max > (1 << 20)) return fail(FMM_ERR_ARG, "batch_max = %d outside [1, 2^20]", batch_max);
    fmm_mlp m = new (std::nothrow) fmm_mlp_s();
    if (!m) return fail(FMM_ERR_OOM, "host allocation");
    if (cudaGetDevice(&m->dev) != cudaSuccess) {
        delete m;
        return fail(FMM_ERR_CUDA, "no CUDA device");
    }
    m->bmax = batch_max;
    const size_t b = (size_t)batch_max;
    bool ok = cudaMalloc((void**)&m->params, 4 * NPAR) == cudaSuccess &&
              cudaMalloc((void**)&m->grads, 4 * NPAR) == cudaSuccess &&
              cudaMalloc((void**)&m->m, 4 * NPAR) == cudaSuccess &&
              cudaMalloc((void**)&m->v, 4 * NPAR) == cudaSuccess &&
              cudaMalloc((void**)&m->h1, 4 * b * D1) == cudaSuccess &&
              cudaMalloc((void**)&m->h2, 4 * b * D2) == cudaSuccess &&
              cudaMalloc((void**)&m->z, 4 * b * D3) == cudaSuccess &&
              cudaMalloc((void**)&m->dz, 4 * b * D3) == cudaSuccess &&
              cudaMalloc((void**)&m->dh2, 4 * b * D2) == cudaSuccess &&
              cudaMalloc((void**)&m->dh1, 4 * b * D1) == cudaSuccess &&
              cudaMalloc((void**)&m->loss, 4 * b) == cudaSuccess &&
              cudaMalloc((void**)&m->lossm, 4) == cudaSuccess;
    if (!ok) {
        free_mlp(m);
        return fail(FMM_ERR_OOM, "network storage");
    }
    if (cudaMemset(m->params, 0, 4 * NPAR) != cudaSuccess || cudaMemset(m->m, 0, 4 * NPAR) != cudaSuccess ||
        cudaMemset(m->v, 0, 4 * NPAR) != cudaSuccess) {
        free_mlp(m);
        return fail(FMM_ERR_CUDA, "memset");
    }
    *out = m;
    return FMM_OK;
}

void fmm_mlp_destroy(fmm_mlp m)
{
    if (!m) return;
    Guard g(m->dev);
    free_mlp(m);
}

int fmm_mlp_set_params(fmm_mlp m, const float* params, void* stream)
{
    if (!m || !params) return fail(FMM_ERR_ARG, "NULL argument");
    Guard g(m->dev);
    cudaStream_t s = (cudaStream_t)stream;
    FMM_CUDA(cudaMemcpyAsync(m->params, params, 4 * NPAR, cudaMemcpyDefault, s));
    FMM_CUDA(cudaMemsetAsync(m->m, 0, 4 * NPAR, s));
    FMM_CUDA(cudaMemsetAsync(m->v, 0, 4 * NPAR, s));
    m->step = 0;
    return FMM_OK;
}

int fmm_mlp_get_params(fmm_mlp m, float* params, void* stream)
{
    if (!m || !params) return fail(FMM_ERR_ARG, "NULL argument");
    Guard g(m->dev);
    FMM_CUDA(cudaMemcpyAsync(params, m->params, 4 * NPAR, cudaMemcpyDefault, (cudaStream_t)stream));
    return FMM_OK;
}

int fmm_mlp_forward(fmm_mlp m, const float* X, int B, float* prob, void* stream)
{
    int rc = check_batch(m, B);
    if (rc) return rc;
    if (!X || !prob) return fail(FMM_ERR_ARG, "NULL argument");
    Guard g(m->dev);
    cudaStream_t s = (cudaStream_t)stream;
    forward(m, X, B, s);
    k_softmax_xent<<<(B + 7) / 8, 256, 0, s>>>(B, m->z, nullptr, nullptr, nullptr); note_launch();
    FMM_CUDA(cudaMemcpyAsync(prob, m->z, 4 * (size_t)B * D3, cudaMemcpyDeviceToDevice, s));
    FMM_LAUNCH_CHECK("mlp: forward");
    return FMM_OK;
}

int fmm_mlp_gradients(fmm_mlp m, const float* X, const int32_t* label, int B, float* grad, float* loss,
                      void* stream)
{
    int rc = check_batch(m, B);
    if (rc) return rc;
    if (!X || !label) return fail(FMM_ERR_ARG, "NULL argument");
    Guard g(m->dev);
    cudaStream_t s = (cudaStream_t)stream;
    rc = grads_and_loss(m, X, label, B, s);
    if (rc) return rc;
    if (grad) FMM_CUDA(cudaMemcpyAsync(grad, m->grads, 4 * NPAR, cudaMemcpyDeviceToDevice, s));
    if (loss) FMM_CUDA(cudaMemcpyAsync(loss, m->lossm, 4, cudaMemcpyDeviceToDevice, s));
    return FMM_OK;
}

int fmm_mlp_train_step(fmm_mlp m, const float* X, const int32_t* label, int B, float lr, float* loss,
                       void* stream)
{
    int rc = check_batch(m, B);
    if (rc) return rc;
    if (!X || !label) return fail(FMM_ERR_ARG, "NULL argument");
    if (!(lr > 0.f)) return fail(FMM_ERR_ARG, "learning rate must be positive");
    Guard g(m->dev);
    cudaStream_t s = (cudaStream_t)stream;
    rc = grads_and_loss(m, X, label, B, s);
    if (rc) return rc;
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)pow((double)b1, (double)m->step), c2 = 1.f - (float)pow((double)b2, (double)m->step);
    k_adam<<<(int)((NPAR + 255) / 256), 256, 0, s>>>(NPAR, m->params, m->grads, m->m, m->v, lr, b1, b2, 1e-8f, c1, c2);
    note_launch();
    FMM_LAUNCH_CHECK("mlp: adam");
    if (loss) FMM_CUDA(cudaMemcpyAsync(loss, m->lossm, 4, cudaMemcpyDeviceToDevice, s));
    return FMM_OK;
}

int fmm_select_params(fmm_mlp m, const float* features, int B, int32_t* levels_p, void* stream)
{
    int rc = check_batch(m, B);
    if (rc) return rc;
    if (!features || !levels_p) return fail(FMM_ERR_ARG, "NULL argument");
    Guard g(m->dev);
    cudaStream_t s = (cudaStream_t)stream;
    forward(m, features, B, s);
    k_softmax_xent<<<(B + 7) / 8, 256, 0, s>>>(B, m->z, nullptr, nullptr, nullptr); note_launch();
    k_select<<<(B + 7) / 8, 256, 0, s>>>(B, m->z, features, levels_p); note_launch();
    FMM_LAUNCH_CHECK("mlp: select");
    return FMM_OK;
}

}  // extern "C"
