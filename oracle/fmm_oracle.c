/*
 * Plain FP64 CPU oracle for the asymmetric adaptive 2D fast multipole method of
 * S. Engblom, "On well-separated sets and fast multipole methods".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or constant with the
 * CUDA library and must never be used as a fallback for it.
 *
 * What it computes (all in IEEE binary64, round to nearest; build with -ffp-contract=off so
 * that the compiler fuses no multiply-add, which keeps the tree and the interaction lists
 * reproducible bit for bit):
 *
 *   Eq. (1.1):  Phi(x_i) = sum_{j != i} G(x_i, x_j) with the 2D harmonic kernel
 *               G(x_i, x_j) = q_j log|x_i - x_j|   (strengths q_j as in Section 5).
 *
 *   - orc_direct : the plain O(N^2) definition of Eq. (1.1) (the reference for every error).
 *   - orc_tree   : the balanced asymmetric mesh of Section 4 / Fig. 1.1 / Fig. 4.1, built by
 *                  recursive median splits along each coordinate direction.
 *   - orc_lists  : the strong/weak connectivity rule of Section 4 with the theta-criterion
 *                  (Criterion 2.1).
 *   - orc_fmm    : the full method -- P2M, M2M, M2L on the weak lists, L2L, L2P and direct
 *                  evaluation on the finest-level strong lists -- using the classical complex
 *                  multipole/local representation that Section 5 names (Greengard & Rokhlin,
 *                  ref. [FMM]); the paper does not print those formulas, so they are written
 *                  out here from their derivation (see the comment above each operator).
 *
 * Readings of points the paper leaves open (each one is also listed in the design notes):
 *   R1  x is split first, then y separately in each x-half; the lower part of a set of n
 *       points gets floor(n/2) of them (Section 4 splits every box close to its median in
 *       both coordinates; Fig. 1.1 shows four boxes holding almost the same counts).
 *   R2  ties in a coordinate are broken by the original input index.
 *   R3  the split coordinate is 0.5*(a+b) of the two straddling coordinates.
 *   R4  the sphere of a box for Criterion 2.1 is the circumscribed circle of its partition
 *       rectangle (Section 2: the representation covers the whole enclosing box).
 *   R5  "<=" in the criterion; in addition the two spheres must be disjoint (the hypothesis of
 *       Criterion 2.1), which only matters when both radii are zero.
 *   R6  p is the order: coefficients k = 0..p (a_0 is the log term).
 *   R7  coincident points contribute nothing (log 0 is skipped, like j = i).
 *   R8  canonical point order: leaves in level order, inside a leaf ascending input index.
 *   R19 parent-level interactions (optional, flags & 1): only four consecutive weak entries
 *       4k .. 4k+3 (all children of one box, in candidate order) are replaced, by one entry for
 *       their parent in the position of the first, when Criterion 2.1 holds for the parent.
 *   R20 role exchange (optional, flags & 2): finest level only; a strong leaf pair passes when
 *       r + theta*R <= theta*d and R + r < d; the smaller target takes P2L, the larger M2P; the
 *       pair leaves the strong list.
 *   R21 the uniform mesh of the comparison (flags & 4): square root on the bounding box's
 *       lower-left corner with the longer side, geometric quadrants, the same lists and
 *       expansions (see orc_tree_uniform).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------------------------
 * Tree: Section 4 (recursive median splits, pyramid storage), Fig. 1.1 and Fig. 4.1.
 * Boxes are numbered in level order: box i of level l has global id (4^l - 1)/3 + i and its
 * children are boxes 4i+k of level l+1, k = 0:(x-low,y-low) 1:(x-low,y-high)
 * 2:(x-high,y-low) 3:(x-high,y-high).
 * ------------------------------------------------------------------------------------------ */

typedef struct { double key; int32_t idx; } keyed;

static int cmp_keyed(const void* a, const void* b)
{
    const keyed* u = (const keyed*)a;
    const keyed* v = (const keyed*)b;
    if (u->key < v->key) return -1;
    if (u->key > v->key) return 1;
    if (u->idx < v->idx) return -1;
    if (u->idx > v->idx) return 1;
    return 0;
}

static int cmp_int32(const void* a, const void* b)
{
    int32_t u = *(const int32_t*)a, v = *(const int32_t*)b;
    return (u > v) - (u < v);
}

/* Order seg[0..m) by (coord, index), lexicographically (reading R2). */
static void sort_by(int32_t* seg, int64_t m, const double* coord, keyed* tmp)
{
    for (int64_t i = 0; i < m; i++) { tmp[i].key = coord[seg[i]]; tmp[i].idx = seg[i]; }
    qsort(tmp, (size_t)m, sizeof(keyed), cmp_keyed);
    for (int64_t i = 0; i < m; i++) seg[i] = tmp[i].idx;
}

int64_t orc_nbox(int L)
{
    int64_t s = 0, w = 1;
    for (int l = 0; l <= L; l++) { s += w; w *= 4; }
    return s;
}

static int64_t level_base(int l) { return ((((int64_t)1) << (2 * l)) - 1) / 3; }

/*
 * Build the tree.  perm[n] (output): canonical point order (reading R8), i.e. perm[k] is the
 * input index of the k-th point.  rects[4*nbox] (output): (x0, x1, y0, y1) per box in level
 * order.  leaf_begin[4^L + 1] (output): leaf i holds perm[leaf_begin[i] .. leaf_begin[i+1]).
 * Returns 0, -1 for bad arguments, -3 when n < 4^L (some leaf would be empty).
 */
int orc_tree(int64_t n, const double* x, const double* y, int L,
             int32_t* perm, double* rects, int64_t* leaf_begin)
{
    if (n <= 0 || L < 0 || L > 15 || !x || !y || !perm || !rects || !leaf_begin) return -1;
    if (n < (((int64_t)1) << (2 * L))) return -3;
    int32_t* work = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    keyed* tmp = (keyed*)malloc(sizeof(keyed) * (size_t)n);
    int64_t nleaf = ((int64_t)1) << (2 * L);
    int64_t* beg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nleaf + 1));
    int64_t* nbeg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nleaf + 1));
    for (int64_t i = 0; i < n; i++) work[i] = (int32_t)i;

    /* root: the tight bounding box of all points */
    double x0 = x[0], x1 = x[0], y0 = y[0], y1 = y[0];
    for (int64_t i = 1; i < n; i++) {
        if (x[i] < x0) x0 = x[i];
        if (x[i] > x1) x1 = x[i];
        if (y[i] < y0) y0 = y[i];
        if (y[i] > y1) y1 = y[i];
    }
    rects[0] = x0; rects[1] = x1; rects[2] = y0; rects[3] = y1;
    beg[0] = 0; beg[1] = n;

    for (int l = 0; l < L; l++) {
        int64_t nb = ((int64_t)1) << (2 * l);
        for (int64_t b = 0; b < nb; b++) {
            int32_t* seg = work + beg[b];
            int64_t m = beg[b + 1] - beg[b];
            /* x-split: the lower floor(m/2) points in (x, index) order form the x-low half */
            sort_by(seg, m, x, tmp);
            int64_t mx = m / 2;
            double xs = 0.5 * (x[seg[mx - 1]] + x[seg[mx]]);
            /* y-split of each half separately */
            int64_t hb[2] = {0, mx}, hn[2] = {mx, m - mx};
            double ys[2];
            int64_t hy[2];
            for (int h = 0; h < 2; h++) {
                int32_t* hs = seg + hb[h];
                sort_by(hs, hn[h], y, tmp);
                hy[h] = hn[h] / 2;
                ys[h] = 0.5 * (y[hs[hy[h] - 1]] + y[hs[hy[h]]]);
            }
            /* children in id order: (xl,yl), (xl,yh), (xh,yl), (xh,yh) */
            nbeg[4 * b + 0] = beg[b];
            nbeg[4 * b + 1] = beg[b] + hy[0];
            nbeg[4 * b + 2] = beg[b] + mx;
            nbeg[4 * b + 3] = beg[b] + mx + hy[1];
            const double* pr = rects + 4 * (level_base(l) + b);
            double* cr = rects + 4 * (level_base(l + 1) + 4 * b);
            double px0 = pr[0], px1 = pr[1], py0 = pr[2], py1 = pr[3];
            cr[0] = px0; cr[1] = xs;  cr[2] = py0;   cr[3] = ys[0];
            cr[4] = px0; cr[5] = xs;  cr[6] = ys[0]; cr[7] = py1;
            cr[8] = xs;  cr[9] = px1; cr[10] = py0;  cr[11] = ys[1];
            cr[12] = xs; cr[13] = px1; cr[14] = ys[1]; cr[15] = py1;
        }
        nbeg[4 * nb] = n;
        memcpy(beg, nbeg, sizeof(int64_t) * (size_t)(4 * nb + 1));
    }
    /* canonical order inside each leaf: ascending input index */
    for (int64_t b = 0; b < nleaf; b++) {
        qsort(work + beg[b], (size_t)(beg[b + 1] - beg[b]), sizeof(int32_t), cmp_int32);
        leaf_begin[b] = beg[b];
    }
    leaf_begin[nleaf] = n;
    memcpy(perm, work, sizeof(int32_t) * (size_t)n);
    free(work); free(tmp); free(beg); free(nbeg);
    return 0;
}

/*
 * The uniform-grid mesh (the classical non-adaptive FMM mesh that Section 5 compares the adaptive
 * one with, reading R21): the root is the square [x0, x0 + s] x [y0, y0 + s] with (x0, y0) the
 * lower-left corner of the points' bounding box and s its longer side; every box splits into
 * four equal quadrants, children numbered as in orc_tree (x-low/y-low, x-low/y-high, x-high/
 * y-low, x-high/y-high).  Cell (ix, iy) of level l has x-range
 * [x0 + s*(ix/2^l), x0 + s*((ix+1)/2^l)], and likewise in y.  A point's leaf has
 * ix = floor(((x - x0) / s) * 2^L), clamped to [0, 2^L - 1] (iy likewise; all 0 when s = 0).
 * Leaves may be empty or hold any number of points.  The canonical order is by leaf, then by
 * input index, and leaf_begin counts the points.  root (may be NULL): a given root square
 * (x0, y0, side) instead of the bounding one, e.g. the unit square of Section 5's experiment.
 * Returns 0, or -1 for bad arguments.
 */
int orc_tree_uniform(int64_t n, const double* x, const double* y, int L, const double* root,
                     int32_t* perm, double* rects, int64_t* leaf_begin)
{
    if (n <= 0 || L < 0 || L > 15 || !x || !y || !perm || !rects || !leaf_begin) return -1;
    double x0 = x[0], x1 = x[0], y0 = y[0], y1 = y[0];
    for (int64_t i = 1; i < n; i++) {
        if (x[i] < x0) x0 = x[i];
        if (x[i] > x1) x1 = x[i];
        if (y[i] < y0) y0 = y[i];
        if (y[i] > y1) y1 = y[i];
    }
    const double sx = x1 - x0, sy = y1 - y0;
    double side = sx > sy ? sx : sy;
    if (root) { /* a given root square (x0, y0, side); points outside fall into its edge cells */
        if (!(root[2] >= 0.0)) return -1;
        x0 = root[0];
        y0 = root[1];
        side = root[2];
    }
    const int64_t nleaf = ((int64_t)1) << (2 * L), m = ((int64_t)1) << L;
    /* every box of every level */
    for (int l = 0; l <= L; l++) {
        const int64_t nb = ((int64_t)1) << (2 * l);
        const double w = (double)(((int64_t)1) << l);
        for (int64_t b = 0; b < nb; b++) {
            int64_t ix = 0, iy = 0;
            for (int j = 0; j < l; j++) { /* digit j (from the top) of b: x bit, y bit */
                const int64_t d = (b >> (2 * (l - 1 - j))) & 3;
                ix = 2 * ix + (d >> 1);
                iy = 2 * iy + (d & 1);
            }
            double* r = rects + 4 * (level_base(l) + b);
            r[0] = x0 + side * ((double)ix / w);
            r[1] = x0 + side * ((double)(ix + 1) / w);
            r[2] = y0 + side * ((double)iy / w);
            r[3] = y0 + side * ((double)(iy + 1) / w);
        }
    }
    /* leaf of every point, then a stable counting sort by leaf */
    int64_t* leaf = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t b = 0; b <= nleaf; b++) leaf_begin[b] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t ix = 0, iy = 0;
        if (side > 0.0) {
            ix = (int64_t)floor(((x[i] - x0) / side) * (double)m);
            iy = (int64_t)floor(((y[i] - y0) / side) * (double)m);
            if (ix > m - 1) ix = m - 1;
            if (iy > m - 1) iy = m - 1;
            if (ix < 0) ix = 0;
            if (iy < 0) iy = 0;
        }
        int64_t id = 0;
        for (int j = L - 1; j >= 0; j--) id = 4 * id + 2 * ((ix >> j) & 1) + ((iy >> j) & 1);
        leaf[i] = id;
        leaf_begin[id + 1]++;
    }
    for (int64_t b = 0; b < nleaf; b++) leaf_begin[b + 1] += leaf_begin[b];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nleaf);
    memcpy(fill, leaf_begin, sizeof(int64_t) * (size_t)nleaf);
    for (int64_t i = 0; i < n; i++) perm[fill[leaf[i]]++] = (int32_t)i;
    free(fill);
    free(leaf);
    return 0;
}

/* Box geometry: centre = midpoint of the rectangle, radius = half its diagonal (reading R4). */
void orc_geometry(int64_t nbox, const double* rects, double* centers, double* radii)
{
    for (int64_t g = 0; g < nbox; g++) {
        const double* r = rects + 4 * g;
        double w = r[1] - r[0], h = r[3] - r[2];
        centers[2 * g] = 0.5 * (r[0] + r[1]);
        centers[2 * g + 1] = 0.5 * (r[2] + r[3]);
        radii[g] = 0.5 * sqrt(w * w + h * h);
    }
}

/*
 * Criterion 2.1 (theta-criterion): spheres (c1, r1), (c2, r2), d = |c1 - c2|,
 * R = max(r1, r2), r = min(r1, r2); well-separated iff R + theta*r <= theta*d, for spheres that
 * are disjoint (R + r < d; reading R5).  Returns 1 when well-separated.
 */
int orc_theta_weak(double c1x, double c1y, double r1, double c2x, double c2y, double r2,
                   double theta)
{
    double dx = c1x - c2x, dy = c1y - c2y;
    double d = sqrt(dx * dx + dy * dy);
    double R = r1 > r2 ? r1 : r2;
    double r = r1 > r2 ? r2 : r1;
    return (R + theta * r <= theta * d) && (R + r < d);
}

/*
 * The same criterion with the roles of the two radii exchanged (Section 4, finest-level
 * optimisation): r + theta*R <= theta*d, i.e. the smaller sphere seen from outside the larger one
 * at ratio <= theta, for disjoint spheres.  Only differs from Criterion 2.1 when r < R.
 */
int orc_theta_swapped(double c1x, double c1y, double r1, double c2x, double c2y, double r2,
                      double theta)
{
    double dx = c1x - c2x, dy = c1y - c2y;
    double d = sqrt(dx * dx + dy * dy);
    double R = r1 > r2 ? r1 : r2;
    double r = r1 > r2 ? r2 : r1;
    return (r + theta * R <= theta * d) && (R + r < d);
}

/* ------------------------------------------------------------------------------------------
 * Connectivity: Section 4.  S(root) = {root}, W(root) = {}.  For a box b on level l >= 1, the
 * candidates are the children of every box in S(parent(b)), taken in ascending id; a candidate
 * that is well-separated from b joins W(b), every other one joins S(b).  A box is always in
 * its own strong list (d = 0 fails the criterion).  Lists hold within-level box indices.
 * ------------------------------------------------------------------------------------------ */

typedef struct {
    int L;
    int64_t nbox;
    int64_t* woff;  /* nbox + 1, global id order */
    int64_t* soff;
    int32_t* widx;
    int32_t* sidx;
    int64_t wcap, scap;
    int64_t* xoff;  /* role-exchange lists of the finest level (NULL unless built) */
    int32_t* xidx;
} orc_lists_t;

static void push(int32_t** a, int64_t* cap, int64_t n, int32_t v)
{
    if (n >= *cap) {
        *cap = *cap ? 2 * *cap : 1024;
        *a = (int32_t*)realloc(*a, sizeof(int32_t) * (size_t)*cap);
    }
    (*a)[n] = v;
}

void* orc_lists_build(int L, const double* rects, double theta)
{
    orc_lists_t* h = (orc_lists_t*)calloc(1, sizeof(orc_lists_t));
    h->L = L;
    h->nbox = orc_nbox(L);
    h->woff = (int64_t*)calloc((size_t)h->nbox + 1, sizeof(int64_t));
    h->soff = (int64_t*)calloc((size_t)h->nbox + 1, sizeof(int64_t));
    double* c = (double*)malloc(sizeof(double) * 2 * (size_t)h->nbox);
    double* r = (double*)malloc(sizeof(double) * (size_t)h->nbox);
    orc_geometry(h->nbox, rects, c, r);
    int64_t nw = 0, ns = 0;
    /* root */
    h->woff[0] = 0; h->soff[0] = 0;
    push(&h->sidx, &h->scap, ns++, 0);
    h->woff[1] = nw; h->soff[1] = ns;
    for (int l = 1; l <= L; l++) {
        int64_t nb = ((int64_t)1) << (2 * l);
        int64_t base = level_base(l), pbase = level_base(l - 1);
        for (int64_t b = 0; b < nb; b++) {
            int64_t g = base + b;
            int64_t pg = pbase + b / 4;
            for (int64_t e = h->soff[pg]; e < h->soff[pg + 1]; e++) {
                int64_t P = h->sidx[e];
                for (int k = 0; k < 4; k++) {
                    int64_t cb = 4 * P + k, cg = base + cb;
                    if (orc_theta_weak(c[2 * g], c[2 * g + 1], r[g],
                                       c[2 * cg], c[2 * cg + 1], r[cg], theta))
                        push(&h->widx, &h->wcap, nw++, (int32_t)cb);
                    else
                        push(&h->sidx, &h->scap, ns++, (int32_t)cb);
                }
            }
            h->woff[g + 1] = nw;
            h->soff[g + 1] = ns;
        }
    }
    free(c); free(r);
    return h;
}

/* Optional structural optimisation of Section 4: when the four children of a box P all sit on a
 * target's weak list and Criterion 2.1 also holds between P and the target, one M2L term from P
 * replaces the four from its children.  The
 * four children appear as four consecutive weak entries 4k, 4k+1, 4k+2, 4k+3 (candidates are
 * taken parent by parent, child by child); they are replaced, in place of the first, by one entry
 * k | ORC_PARENT_FLAG naming the parent at the level above.  Applied once to every level's weak
 * lists after they are complete (the strong lists, which generate the next level's candidates,
 * are untouched). */
#define ORC_PARENT_FLAG 0x40000000

void orc_lists_merge_parents(void* hp, const double* rects, double theta)
{
    orc_lists_t* h = (orc_lists_t*)hp;
    double* c = (double*)malloc(sizeof(double) * 2 * (size_t)h->nbox);
    double* r = (double*)malloc(sizeof(double) * (size_t)h->nbox);
    orc_geometry(h->nbox, rects, c, r);
    int64_t* noff = (int64_t*)calloc((size_t)h->nbox + 1, sizeof(int64_t));
    int32_t* nidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(h->woff[h->nbox] + 1));
    int64_t nw = 0;
    for (int64_t g = 0; g < h->nbox; g++) {
        noff[g] = nw;
        int l = 0;
        while (level_base(l + 1) <= g) l++;
        const int64_t pbase = l >= 1 ? level_base(l - 1) : 0;
        int64_t e = h->woff[g];
        while (e < h->woff[g + 1]) {
            const int32_t v = h->widx[e];
            if (l >= 1 && e + 3 < h->woff[g + 1] && v % 4 == 0 && h->widx[e + 1] == v + 1 &&
                h->widx[e + 2] == v + 2 && h->widx[e + 3] == v + 3) {
                const int64_t P = pbase + v / 4;
                if (orc_theta_weak(c[2 * g], c[2 * g + 1], r[g], c[2 * P], c[2 * P + 1], r[P], theta)) {
                    nidx[nw++] = (v / 4) | ORC_PARENT_FLAG;
                    e += 4;
                    continue;
                }
            }
            nidx[nw++] = v;
            e++;
        }
    }
    noff[h->nbox] = nw;
    free(h->woff);
    free(h->widx);
    h->woff = noff;
    h->widx = nidx;
    h->wcap = h->woff[h->nbox] + 1;
    free(c); free(r);
}

/* The second optional optimisation of Section 4, at the finest level only: a strongly coupled
 * pair of leaves of different radii whose criterion holds with the roles of r and R exchanged
 * (orc_theta_swapped) is taken out of the strong list of the target leaf and put on its role
 * exchange list X, in the same order.  If the target is the smaller leaf, the source's points
 * become terms of the target's local expansion (P2L); if it is the larger one, the source's
 * multipole expansion is evaluated at the target's points (M2P) and the entry carries
 * ORC_SWAP_M2P.  Applied once, after the lists are complete. */
#define ORC_SWAP_M2P 0x20000000

void orc_lists_swap_leaves(void* hp, const double* rects, double theta)
{
    orc_lists_t* h = (orc_lists_t*)hp;
    double* c = (double*)malloc(sizeof(double) * 2 * (size_t)h->nbox);
    double* r = (double*)malloc(sizeof(double) * (size_t)h->nbox);
    orc_geometry(h->nbox, rects, c, r);
    const int64_t base = level_base(h->L);
    int64_t* nsoff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(h->nbox + 1));
    int32_t* nsidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(h->soff[h->nbox] + 1));
    h->xoff = (int64_t*)calloc((size_t)h->nbox + 1, sizeof(int64_t));
    h->xidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(h->soff[h->nbox] + 1));
    int64_t ns = 0, nx = 0;
    for (int64_t g = 0; g < h->nbox; g++) {
        nsoff[g] = ns;
        h->xoff[g] = nx;
        for (int64_t e = h->soff[g]; e < h->soff[g + 1]; e++) {
            const int32_t v = h->sidx[e];
            const int64_t sg = base + v;
            if (g >= base &&
                orc_theta_swapped(c[2 * g], c[2 * g + 1], r[g], c[2 * sg], c[2 * sg + 1], r[sg], theta))
                h->xidx[nx++] = r[g] > r[sg] ? (v | ORC_SWAP_M2P) : v;
            else
                nsidx[ns++] = v;
        }
    }
    nsoff[h->nbox] = ns;
    h->xoff[h->nbox] = nx;
    free(h->soff);
    free(h->sidx);
    h->soff = nsoff;
    h->sidx = nsidx;
    h->scap = ns + 1;
    free(c); free(r);
}

/* kind: 1 weak, 0 strong, 2 role exchange (empty unless orc_lists_swap_leaves ran) */
int64_t orc_lists_total(void* hp, int kind)
{
    orc_lists_t* h = (orc_lists_t*)hp;
    if (kind == 2) return h->xoff ? h->xoff[h->nbox] : 0;
    return kind ? h->woff[h->nbox] : h->soff[h->nbox];
}

void orc_lists_copy(void* hp, int kind, int64_t* off, int32_t* idx)
{
    orc_lists_t* h = (orc_lists_t*)hp;
    if (kind == 2 && !h->xoff) {
        memset(off, 0, sizeof(int64_t) * (size_t)(h->nbox + 1));
        return;
    }
    const int64_t* o = kind == 2 ? h->xoff : kind ? h->woff : h->soff;
    const int32_t* v = kind == 2 ? h->xidx : kind ? h->widx : h->sidx;
    memcpy(off, o, sizeof(int64_t) * (size_t)(h->nbox + 1));
    if (o[h->nbox]) memcpy(idx, v, sizeof(int32_t) * (size_t)o[h->nbox]);
}

void orc_lists_free(void* hp)
{
    orc_lists_t* h = (orc_lists_t*)hp;
    if (!h) return;
    free(h->woff); free(h->soff); free(h->widx); free(h->sidx); free(h->xoff); free(h->xidx); free(h);
}

/* ------------------------------------------------------------------------------------------
 * Expansions: the classical complex representation (Section 5, refs. [FMM, AFMM]), unscaled.
 * With z a point of the complex plane, the potential of unit strength at z_j is
 * Re log(z - z_j) = log|z - z_j|.
 *
 * Multipole about c:  phi(z) = a_0 log(z - c) + sum_{k=1..p} a_k (z - c)^{-k},
 *                      a_0 = sum q_j,  a_k = -sum q_j (z_j - c)^k / k      (since
 *                      log(z - z_j) = log(z - c) - sum_k ((z_j - c)/(z - c))^k / k).
 * Local about c:       psi(z) = sum_{l=0..p} b_l (z - c)^l.
 * Binomials C(n, k) come from Pascal's triangle in double precision.
 * ------------------------------------------------------------------------------------------ */

#define ORC_PMAX 64
static double binom_tab[2 * ORC_PMAX + 2][2 * ORC_PMAX + 2];
static int binom_ready = 0;

static double binom(int n, int k)
{
    if (!binom_ready) {
        for (int i = 0; i < 2 * ORC_PMAX + 2; i++) {
            binom_tab[i][0] = 1.0;
            for (int j = 1; j <= i; j++)
                binom_tab[i][j] = binom_tab[i - 1][j - 1] + (j <= i - 1 ? binom_tab[i - 1][j] : 0.0);
        }
        binom_ready = 1;
    }
    if (k < 0 || k > n || n < 0) return 0.0;
    return binom_tab[n][k];
}

/* P2M: multipole coefficients a[0..p] about c of sources (x_j, y_j, q_j). */
static void p2m(int64_t m, const int32_t* ids, const double* x, const double* y, const double* q,
                cplx c, int p, cplx* a)
{
    for (int k = 0; k <= p; k++) a[k] = 0;
    for (int64_t t = 0; t < m; t++) {
        int64_t j = ids ? ids[t] : t;
        cplx dz = (x[j] + I * y[j]) - c;
        cplx pw = 1.0;
        a[0] += q[j];
        for (int k = 1; k <= p; k++) {
            pw *= dz;
            a[k] -= q[j] * pw / (double)k;
        }
    }
}

/*
 * M2M: shift a multipole from a child centre to the parent centre, z0 = c_child - c_parent.
 * With w = z - c_parent:  log(w - z0) = log w - sum_l (z0/w)^l / l  and
 * (w - z0)^{-k} = sum_{l>=k} C(l-1, k-1) z0^{l-k} w^{-l}, so
 *   b_0 = a_0,   b_l = -a_0 z0^l / l + sum_{k=1..l} a_k C(l-1, k-1) z0^{l-k}.
 * Accumulates into b.
 */
static void m2m(const cplx* a, cplx z0, int p, cplx* b)
{
    cplx zp[ORC_PMAX + 1];
    zp[0] = 1.0;
    for (int l = 1; l <= p; l++) zp[l] = zp[l - 1] * z0;
    b[0] += a[0];
    for (int l = 1; l <= p; l++) {
        cplx s = -a[0] * zp[l] / (double)l;
        for (int k = 1; k <= l; k++) s += a[k] * binom(l - 1, k - 1) * zp[l - k];
        b[l] += s;
    }
}

/*
 * M2L: convert a multipole about c_src into a local expansion about c_tgt, z0 = c_src - c_tgt.
 * With w = z - c_tgt:  log(w - z0) = log(-z0) - sum_l (w/z0)^l / l  and
 * (w - z0)^{-k} = (-1)^k z0^{-k} sum_{l>=0} C(l+k-1, k-1) (w/z0)^l, so
 *   b_0 = a_0 log(-z0) + sum_k a_k (-1)^k z0^{-k},
 *   b_l = -a_0 / (l z0^l) + z0^{-l} sum_k a_k (-1)^k C(l+k-1, k-1) z0^{-k}.
 * Accumulates into b.
 */
static void m2l(const cplx* a, cplx z0, int p, cplx* b)
{
    cplx iz[2 * ORC_PMAX + 2];
    iz[0] = 1.0;
    cplx inv = 1.0 / z0;
    for (int k = 1; k <= 2 * p; k++) iz[k] = iz[k - 1] * inv;
    cplx s0 = a[0] * clog(-z0);
    for (int k = 1; k <= p; k++) s0 += a[k] * ((k & 1) ? -1.0 : 1.0) * iz[k];
    b[0] += s0;
    for (int l = 1; l <= p; l++) {
        cplx s = -a[0] / (double)l;
        for (int k = 1; k <= p; k++)
            s += a[k] * ((k & 1) ? -1.0 : 1.0) * binom(l + k - 1, k - 1) * iz[k];
        b[l] += s * iz[l];
    }
}

/*
 * L2L: re-centre a local expansion from c_parent to c_child, z0 = c_child - c_parent.
 * (w + z0)^k = sum_{l<=k} C(k, l) w^l z0^{k-l}, so  b'_l = sum_{k=l..p} b_k C(k, l) z0^{k-l}.
 * Accumulates into out.
 */
static void l2l(const cplx* b, cplx z0, int p, cplx* out)
{
    cplx zp[ORC_PMAX + 1];
    zp[0] = 1.0;
    for (int l = 1; l <= p; l++) zp[l] = zp[l - 1] * z0;
    for (int l = 0; l <= p; l++) {
        cplx s = 0;
        for (int k = l; k <= p; k++) s += b[k] * binom(k, l) * zp[k - l];
        out[l] += s;
    }
}

/* L2P: Re sum_l b_l dz^l with dz = z - c. */
static double l2p(const cplx* b, cplx dz, int p)
{
    cplx s = 0, pw = 1.0;
    for (int l = 0; l <= p; l++) { s += b[l] * pw; pw *= dz; }
    return creal(s);
}

/* Derivative of the local expansion: sum_{l >= 1} l b_l dz^(l-1), dz = z - c. */
static cplx l2p_deriv(const cplx* b, cplx dz, int p)
{
    cplx s = 0, pw = 1.0;
    for (int l = 1; l <= p; l++) { s += (double)l * b[l] * pw; pw *= dz; }
    return s;
}

/* M2P: Re[a_0 log(dz) + sum_k a_k dz^{-k}], dz = z - c (the multipole evaluated at a point;
 * used by the role exchange of Section 4). */
static double m2p(const cplx* a, cplx dz, int p)
{
    cplx s = a[0] * clog(dz), pw = 1.0, inv = 1.0 / dz;
    for (int k = 1; k <= p; k++) { pw *= inv; s += a[k] * pw; }
    return creal(s);
}

/* Derivative of the multipole expansion in z: a_0 / dz - sum_k k a_k dz^{-k-1}. */
static cplx m2p_deriv(const cplx* a, cplx dz, int p)
{
    cplx inv = 1.0 / dz, pw = inv, s = a[0] * inv;
    for (int k = 1; k <= p; k++) { pw *= inv; s -= (double)k * a[k] * pw; }
    return s;
}

/*
 * P2L: the local expansion about c of sources z_j lying outside a disc about c that holds the
 * evaluation points (the role exchange of Section 4).  With w = z - c,
 *   log(z - z_j) = log(c - z_j) + log(1 - w / (z_j - c)) = log(c - z_j) - sum_{l>=1} (w/(z_j - c))^l / l,
 * so b_0 += q_j log(c - z_j) and b_l += -q_j / (l (z_j - c)^l).  Accumulates into b.
 */
static void p2l(int64_t m, const int32_t* ids, const double* x, const double* y, const double* q,
                cplx c, int p, cplx* b)
{
    for (int64_t t = 0; t < m; t++) {
        int64_t j = ids ? ids[t] : t;
        cplx dz = (x[j] + I * y[j]) - c;
        cplx inv = 1.0 / dz, pw = 1.0;
        b[0] += q[j] * clog(-dz);
        for (int l = 1; l <= p; l++) {
            pw *= inv;
            b[l] -= q[j] * pw / (double)l;
        }
    }
}

/* ---- flat-array wrappers of the operators (complex numbers interleaved re, im) ---- */

void orc_p2m(int64_t m, const double* x, const double* y, const double* q, double cx, double cy,
             int p, double* a_out)
{
    cplx a[ORC_PMAX + 1];
    p2m(m, NULL, x, y, q, cx + I * cy, p, a);
    for (int k = 0; k <= p; k++) { a_out[2 * k] = creal(a[k]); a_out[2 * k + 1] = cimag(a[k]); }
}

/* P2L of m sources about (cx, cy); b_out receives the p+1 local coefficients. */
void orc_p2l(int64_t m, const double* x, const double* y, const double* q, double cx, double cy,
             int p, double* b_out)
{
    cplx b[ORC_PMAX + 1];
    for (int l = 0; l <= p; l++) b[l] = 0;
    p2l(m, NULL, x, y, q, cx + I * cy, p, b);
    for (int l = 0; l <= p; l++) { b_out[2 * l] = creal(b[l]); b_out[2 * l + 1] = cimag(b[l]); }
}

static void load_c(const double* v, int p, cplx* c)
{
    for (int k = 0; k <= p; k++) c[k] = v[2 * k] + I * v[2 * k + 1];
}

static void store_c(const cplx* c, int p, double* v)
{
    for (int k = 0; k <= p; k++) { v[2 * k] = creal(c[k]); v[2 * k + 1] = cimag(c[k]); }
}

void orc_m2m(const double* a_in, double zx, double zy, int p, double* b_out)
{
    cplx a[ORC_PMAX + 1], b[ORC_PMAX + 1];
    load_c(a_in, p, a);
    for (int k = 0; k <= p; k++) b[k] = 0;
    m2m(a, zx + I * zy, p, b);
    store_c(b, p, b_out);
}

void orc_m2l(const double* a_in, double zx, double zy, int p, double* b_out)
{
    cplx a[ORC_PMAX + 1], b[ORC_PMAX + 1];
    load_c(a_in, p, a);
    for (int k = 0; k <= p; k++) b[k] = 0;
    m2l(a, zx + I * zy, p, b);
    store_c(b, p, b_out);
}

void orc_l2l(const double* b_in, double zx, double zy, int p, double* b_out)
{
    cplx b[ORC_PMAX + 1], o[ORC_PMAX + 1];
    load_c(b_in, p, b);
    for (int k = 0; k <= p; k++) o[k] = 0;
    l2l(b, zx + I * zy, p, o);
    store_c(o, p, b_out);
}

double orc_l2p(const double* b_in, double dx, double dy, int p)
{
    cplx b[ORC_PMAX + 1];
    load_c(b_in, p, b);
    return l2p(b, dx + I * dy, p);
}

double orc_m2p(const double* a_in, double dx, double dy, int p)
{
    cplx a[ORC_PMAX + 1];
    load_c(a_in, p, a);
    return m2p(a, dx + I * dy, p);
}

/* ------------------------------------------------------------------------------------------
 * Direct summation, Eq. (1.1): phi[t] = sum_{j != tgt[t]} q_j log|x_tgt - x_j|, skipping
 * coincident points (reading R7).  Targets are input indices; threads split the targets.
 * ------------------------------------------------------------------------------------------ */
void orc_direct(int64_t n, const double* x, const double* y, const double* q,
                int64_t m, const int64_t* tgt, double* phi, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t t = 0; t < m; t++) {
        int64_t i = tgt[t];
        double s = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = x[i] - x[j], dy = y[i] - y[j];
            if (dx == 0.0 && dy == 0.0) continue;
            s += q[j] * log(hypot(dx, dy));
        }
        phi[t] = s;
    }
    (void)nthreads;
}

/* ------------------------------------------------------------------------------------------
 * Direct summation of the complex field of Section 5's first experiment,
 * G(z_i, z_j) = -q_j / (z_i - z_j):  F[t] = sum_{j != tgt[t]} -q_j / (z_tgt - z_j), skipping
 * coincident points.  fre/fim receive the real and imaginary parts.
 * ------------------------------------------------------------------------------------------ */
void orc_direct_field(int64_t n, const double* x, const double* y, const double* q,
                      int64_t m, const int64_t* tgt, double* fre, double* fim, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t t = 0; t < m; t++) {
        int64_t i = tgt[t];
        cplx s = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = x[i] - x[j], dy = y[i] - y[j];
            if (dx == 0.0 && dy == 0.0) continue;
            s -= q[j] / (dx + I * dy);
        }
        fre[t] = creal(s);
        fim[t] = cimag(s);
    }
    (void)nthreads;
}

/* ------------------------------------------------------------------------------------------
 * The full method (Section 4):  tree -> connectivity -> upward pass (P2M at the finest level,
 * M2M towards the root) -> M2L along the weak lists of every level -> downward pass (L2L) ->
 * L2P plus direct evaluation along the strong lists of the finest level.  phi is written in
 * input order.  Optional outputs (NULL to skip): the multipole and local coefficients of all
 * boxes, mpole[nbox][p+1] and local[nbox][p+1] as interleaved complex numbers (unscaled, about
 * each box centre; a box's local expansion is complete, i.e. includes its ancestors' shifts).
 * Returns 0 or a negative code as orc_tree.
 * ------------------------------------------------------------------------------------------ */
static int fmm_core(int64_t n, const double* x, const double* y, const double* q, int L, int p,
                    double theta, int flags, const double* root, double* phi, double* fre, double* fim,
                    double* mpole_out, double* local_out)
{
    if (p < 0 || p > ORC_PMAX || !(theta > 0.0 && theta < 1.0)) return -1;
    int64_t nbox = orc_nbox(L), nleaf = ((int64_t)1) << (2 * L);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* rects = (double*)malloc(sizeof(double) * 4 * (size_t)nbox);
    int64_t* lb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nleaf + 1));
    int rc = (flags & 4) ? orc_tree_uniform(n, x, y, L, root, perm, rects, lb) : orc_tree(n, x, y, L, perm, rects, lb);
    if (rc) { free(perm); free(rects); free(lb); return rc; }
    double* cen = (double*)malloc(sizeof(double) * 2 * (size_t)nbox);
    double* rad = (double*)malloc(sizeof(double) * (size_t)nbox);
    orc_geometry(nbox, rects, cen, rad);
    orc_lists_t* li = (orc_lists_t*)orc_lists_build(L, rects, theta);
    if (flags & 1) orc_lists_merge_parents(li, rects, theta);
    if (flags & 2) orc_lists_swap_leaves(li, rects, theta);
    int P = p + 1;
    cplx* M = (cplx*)calloc((size_t)(nbox * P), sizeof(cplx));
    cplx* Lc = (cplx*)calloc((size_t)(nbox * P), sizeof(cplx));
#define CEN(g) (cen[2 * (g)] + I * cen[2 * (g) + 1])

    /* upward pass: P2M on the leaves, then M2M level by level towards the root */
    int64_t lbase = level_base(L);
    for (int64_t b = 0; b < nleaf; b++)
        p2m(lb[b + 1] - lb[b], perm + lb[b], x, y, q, CEN(lbase + b), p, M + (lbase + b) * P);
    for (int l = L - 1; l >= 0; l--) {
        int64_t nb = ((int64_t)1) << (2 * l), base = level_base(l), cbase = level_base(l + 1);
        for (int64_t b = 0; b < nb; b++)
            for (int k = 0; k < 4; k++) {
                int64_t cg = cbase + 4 * b + k;
                m2m(M + cg * P, CEN(cg) - CEN(base + b), p, M + (base + b) * P);
            }
    }
    /* far field: M2L along the weak lists of each level, then L2L to the next level */
    for (int l = 1; l <= L; l++) {
        int64_t nb = ((int64_t)1) << (2 * l), base = level_base(l);
        for (int64_t b = 0; b < nb; b++) {
            int64_t g = base + b;
            for (int64_t e = li->woff[g]; e < li->woff[g + 1]; e++) {
                const int32_t v = li->widx[e];
                int64_t sg = (v & ORC_PARENT_FLAG) ? level_base(l - 1) + (v & ~ORC_PARENT_FLAG) : base + v;
                m2l(M + sg * P, CEN(sg) - CEN(g), p, Lc + g * P);
            }
        }
        if (l < L) {
            int64_t cbase = level_base(l + 1);
            for (int64_t b = 0; b < nb; b++)
                for (int k = 0; k < 4; k++) {
                    int64_t cg = cbase + 4 * b + k;
                    l2l(Lc + (base + b) * P, CEN(cg) - CEN(base + b), p, Lc + cg * P);
                }
        }
    }
    /* role exchange (flags & 2): the sources of a larger leaf on a smaller target's X list join
     * the target's local expansion (P2L) */
    if (li->xoff)
        for (int64_t b = 0; b < nleaf; b++) {
            int64_t g = lbase + b;
            for (int64_t e = li->xoff[g]; e < li->xoff[g + 1]; e++) {
                const int32_t v = li->xidx[e];
                if (v & ORC_SWAP_M2P) continue;
                p2l(lb[v + 1] - lb[v], perm + lb[v], x, y, q, CEN(g), p, Lc + g * P);
            }
        }
    /* evaluation on the finest level: L2P plus direct sums over the strong lists (and, with the
     * role exchange, the multipoles of the smaller leaves on the X list evaluated directly) */
    for (int64_t b = 0; b < nleaf; b++) {
        int64_t g = lbase + b;
        const int64_t x0 = li->xoff ? li->xoff[g] : 0, x1 = li->xoff ? li->xoff[g + 1] : 0;
        for (int64_t t = lb[b]; t < lb[b + 1]; t++) {
            int64_t i = perm[t];
            const cplx zi = x[i] + I * y[i];
            if (fre) {
                /* the field: minus the derivative of the local expansion, minus the near sum */
                cplx f = -l2p_deriv(Lc + g * P, zi - CEN(g), p);
                for (int64_t e = x0; e < x1; e++) {
                    const int32_t v = li->xidx[e];
                    if (!(v & ORC_SWAP_M2P)) continue;
                    const int64_t sg = lbase + (v & ~ORC_SWAP_M2P);
                    f -= m2p_deriv(M + sg * P, zi - CEN(sg), p);
                }
                for (int64_t e = li->soff[g]; e < li->soff[g + 1]; e++) {
                    int64_t sb = li->sidx[e];
                    for (int64_t u = lb[sb]; u < lb[sb + 1]; u++) {
                        int64_t j = perm[u];
                        if (j == i) continue;
                        double dx = x[i] - x[j], dy = y[i] - y[j];
                        if (dx == 0.0 && dy == 0.0) continue;
                        f -= q[j] / (dx + I * dy);
                    }
                }
                fre[i] = creal(f);
                fim[i] = cimag(f);
                continue;
            }
            double s = l2p(Lc + g * P, zi - CEN(g), p);
            for (int64_t e = x0; e < x1; e++) {
                const int32_t v = li->xidx[e];
                if (!(v & ORC_SWAP_M2P)) continue;
                const int64_t sg = lbase + (v & ~ORC_SWAP_M2P);
                s += m2p(M + sg * P, zi - CEN(sg), p);
            }
            for (int64_t e = li->soff[g]; e < li->soff[g + 1]; e++) {
                int64_t sb = li->sidx[e];
                for (int64_t u = lb[sb]; u < lb[sb + 1]; u++) {
                    int64_t j = perm[u];
                    if (j == i) continue;
                    double dx = x[i] - x[j], dy = y[i] - y[j];
                    if (dx == 0.0 && dy == 0.0) continue;
                    s += q[j] * log(hypot(dx, dy));
                }
            }
            phi[i] = s;
        }
    }
#undef CEN
    if (mpole_out)
        for (int64_t e = 0; e < nbox * P; e++) { mpole_out[2 * e] = creal(M[e]); mpole_out[2 * e + 1] = cimag(M[e]); }
    if (local_out)
        for (int64_t e = 0; e < nbox * P; e++) { local_out[2 * e] = creal(Lc[e]); local_out[2 * e + 1] = cimag(Lc[e]); }
    free(M); free(Lc); free(cen); free(rad); free(perm); free(rects); free(lb);
    orc_lists_free(li);
    return 0;
}

int orc_fmm(int64_t n, const double* x, const double* y, const double* q, int L, int p,
            double theta, double* phi, double* mpole_out, double* local_out)
{
    return fmm_core(n, x, y, q, L, p, theta, 0, NULL, phi, NULL, NULL, mpole_out, local_out);
}

/* The method with the optional structural optimisations of Section 4: flags & 1 parent-level
 * interactions (orc_lists_merge_parents), flags & 2 the finest-level role exchange
 * (orc_lists_swap_leaves); flags & 4 runs it on the uniform-grid mesh (orc_tree_uniform)
 * instead of the adaptive one. */
int orc_fmm_ex(int64_t n, const double* x, const double* y, const double* q, int L, int p,
               double theta, int flags, double* phi)
{
    return fmm_core(n, x, y, q, L, p, theta, flags, NULL, phi, NULL, NULL, NULL, NULL);
}

/* The same with the uniform-grid mesh on a given root square (flags & 4; root = x0, y0, side). */
int orc_fmm_root(int64_t n, const double* x, const double* y, const double* q, int L, int p,
                 double theta, int flags, const double* root, double* phi)
{
    return fmm_core(n, x, y, q, L, p, theta, flags | 4, root, phi, NULL, NULL, NULL, NULL);
}

/* The method for the complex field G(z_i, z_j) = -q_j / (z_i - z_j) (Section 5): the same tree,
 * lists and expansions; at the finest level minus the derivative of the local expansion plus the
 * direct field along the strong lists.  fre/fim in input order. */
int orc_fmm_field(int64_t n, const double* x, const double* y, const double* q, int L, int p,
                  double theta, double* fre, double* fim)
{
    return fmm_core(n, x, y, q, L, p, theta, 0, NULL, NULL, fre, fim, NULL, NULL);
}

/* The field with the optional optimisations (flags as orc_fmm_ex). */
int orc_fmm_field_ex(int64_t n, const double* x, const double* y, const double* q, int L, int p,
                     double theta, int flags, double* fre, double* fim)
{
    return fmm_core(n, x, y, q, L, p, theta, flags, NULL, NULL, fre, fim, NULL, NULL);
}
