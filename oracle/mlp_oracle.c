/*
 * FP64 reference of the parameter selector: its input features and its network.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as fmm_oracle.c): loaded by the test suite alone, shares
 * no code, header, table or constant with the CUDA library.
 *
 * The paper fixes the method's parameters by rule (end of Section 4: p ~ log TOL / log theta
 * from Section 3, about 20 points per leaf); the selector learns them instead.  What it computes
 * is defined here from scratch, plainly:
 *
 *   features (64 values): for every level l = 1..15 of a median-split tree (boxes are the
 *     partition rectangles of Section 4), over the 4^l boxes of the level, with long side
 *     s = max(w, h) and short side t = max(min(w, h), 2^-30 s):
 *        mean log2(s / s_root),  standard deviation of log2 s  (population),
 *        mean log2(s / t),       max log2(s / t);
 *     zeros for levels beyond the tree; then log10 N, log10 tol, L / 16, 0.
 *
 *   network: h1 = relu(W1 x + b1) (128), h2 = relu(W2 h1 + b2) (128), z = W3 h2 + b3 (225),
 *     p = softmax(z); loss = mean over the batch of -log p[label].  Parameters in one array:
 *     W1[128][64], b1[128], W2[128][128], b2[128], W3[225][128], b3[225] (row-major).
 *     The gradient is the textbook backward pass of that composition (chain rule, written out
 *     layer by layer below).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NI 64
#define NH 128
#define NO 225

static const long O_W1 = 0;
static const long O_B1 = (long)NH * NI;
static const long O_W2 = (long)NH * NI + NH;
static const long O_B2 = (long)NH * NI + NH + (long)NH * NH;
static const long O_W3 = (long)NH * NI + NH + (long)NH * NH + NH;
static const long O_B3 = (long)NH * NI + NH + (long)NH * NH + NH + (long)NO * NH;

long orc_mlp_nparams(void) { return O_B3 + NO; }

/* y[o] = b[o] + sum_i W[o][i] x[i] */
static void affine(const double* W, const double* b, const double* x, int nin, int nout, double* y)
{
    for (int o = 0; o < nout; o++) {
        double s = b[o];
        for (int i = 0; i < nin; i++) s += W[(long)o * nin + i] * x[i];
        y[o] = s;
    }
}

static void softmax(const double* z, int n, double* p)
{
    double mx = z[0];
    for (int j = 1; j < n; j++)
        if (z[j] > mx) mx = z[j];
    double s = 0;
    for (int j = 0; j < n; j++) {
        p[j] = exp(z[j] - mx);
        s += p[j];
    }
    for (int j = 0; j < n; j++) p[j] /= s;
}

/* prob[B][225] for inputs X[B][64] */
void orc_mlp_forward(const double* prm, const double* X, int B, double* prob)
{
    double a1[NH], h1[NH], a2[NH], h2[NH], z[NO];
    for (int b = 0; b < B; b++) {
        affine(prm + O_W1, prm + O_B1, X + (long)b * NI, NI, NH, a1);
        for (int i = 0; i < NH; i++) h1[i] = a1[i] > 0 ? a1[i] : 0;
        affine(prm + O_W2, prm + O_B2, h1, NH, NH, a2);
        for (int i = 0; i < NH; i++) h2[i] = a2[i] > 0 ? a2[i] : 0;
        affine(prm + O_W3, prm + O_B3, h2, NH, NO, z);
        softmax(z, NO, prob + (long)b * NO);
    }
}

/* mean cross-entropy over the batch; grad (nparams) receives its gradient */
double orc_mlp_loss_grad(const double* prm, const double* X, const int* label, int B, double* grad)
{
    const long np = orc_mlp_nparams();
    memset(grad, 0, sizeof(double) * np);
    double a1[NH], h1[NH], a2[NH], h2[NH], z[NO], p[NO], dz[NO], dh2[NH], dh1[NH];
    double loss = 0;
    for (int b = 0; b < B; b++) {
        const double* x = X + (long)b * NI;
        affine(prm + O_W1, prm + O_B1, x, NI, NH, a1);
        for (int i = 0; i < NH; i++) h1[i] = a1[i] > 0 ? a1[i] : 0;
        affine(prm + O_W2, prm + O_B2, h1, NH, NH, a2);
        for (int i = 0; i < NH; i++) h2[i] = a2[i] > 0 ? a2[i] : 0;
        affine(prm + O_W3, prm + O_B3, h2, NH, NO, z);
        softmax(z, NO, p);
        const int y = label[b];
        loss += -log(p[y]);
        /* d(loss_b / B) / dz = (p - e_y) / B */
        for (int j = 0; j < NO; j++) dz[j] = (p[j] - (j == y ? 1.0 : 0.0)) / B;
        /* layer 3: z = W3 h2 + b3 */
        for (int o = 0; o < NO; o++) {
            grad[O_B3 + o] += dz[o];
            for (int i = 0; i < NH; i++) grad[O_W3 + (long)o * NH + i] += dz[o] * h2[i];
        }
        for (int i = 0; i < NH; i++) {
            double s = 0;
            for (int o = 0; o < NO; o++) s += prm[O_W3 + (long)o * NH + i] * dz[o];
            dh2[i] = a2[i] > 0 ? s : 0; /* through the ReLU */
        }
        /* layer 2: a2 = W2 h1 + b2 */
        for (int o = 0; o < NH; o++) {
            grad[O_B2 + o] += dh2[o];
            for (int i = 0; i < NH; i++) grad[O_W2 + (long)o * NH + i] += dh2[o] * h1[i];
        }
        for (int i = 0; i < NH; i++) {
            double s = 0;
            for (int o = 0; o < NH; o++) s += prm[O_W2 + (long)o * NH + i] * dh2[o];
            dh1[i] = a1[i] > 0 ? s : 0;
        }
        /* layer 1: a1 = W1 x + b1 */
        for (int o = 0; o < NH; o++) {
            grad[O_B1 + o] += dh1[o];
            for (int i = 0; i < NI; i++) grad[O_W1 + (long)o * NI + i] += dh1[o] * x[i];
        }
    }
    return loss / B;
}

/* Features of a tree with L levels over n points: rects in level order (4 per box:
 * x0, x1, y0, y1), out[64]. */
void orc_features(const double* rects, int L, int64_t n, double tol, double* out)
{
    memset(out, 0, sizeof(double) * NI);
    const double* root = rects;
    double sroot = fmax(root[1] - root[0], root[3] - root[2]);
    if (!(sroot > 1e-300)) sroot = 1e-300;
    for (int l = 1; l <= 15 && l <= L; l++) {
        const int64_t nb = (int64_t)1 << (2 * l);
        const int64_t base = (((int64_t)1 << (2 * l)) - 1) / 3;
        double m = 0, m2 = 0, a = 0, amax = 0;
        for (int64_t b = 0; b < nb; b++) {
            const double* r = rects + 4 * (base + b);
            const double w = r[1] - r[0], h = r[3] - r[2];
            double s = w > h ? w : h;
            if (!(s > 1e-300)) s = 1e-300;
            double t = w < h ? w : h;
            if (t < s * ldexp(1.0, -30)) t = s * ldexp(1.0, -30);
            const double ls = log2(s / sroot);
            m += ls;
            m2 += ls * ls;
            const double la = log2(s / t);
            a += la;
            if (la > amax) amax = la;
        }
        const double mean = m / nb;
        double var = m2 / nb - mean * mean;
        if (var < 0) var = 0;
        out[4 * (l - 1) + 0] = mean;
        out[4 * (l - 1) + 1] = sqrt(var);
        out[4 * (l - 1) + 2] = a / nb;
        out[4 * (l - 1) + 3] = amax;
    }
    out[60] = log10((double)n);
    out[61] = log10(tol);
    out[62] = L / 16.0;
    out[63] = 0;
}
