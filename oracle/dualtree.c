/*
 * The paper's own approximations of the leave-one-out score (Holmes, Gray &
 * Isbell, Sec. 3.1-3.4) as a single-threaded CPU reference for accuracy and
 * speed context: the exact GPU path replaces them, so this is prior art kept
 * for comparison, not a reference result (the exact oracle is oracle.c).
 * TEST INFRASTRUCTURE ONLY: tests and the benchmark's context line call it;
 * the product library never does, and nothing here is shared with it.
 *
 * Score: Eq. 3 in the form of Sec. 3.2, L = (1/n) sum_i ln A_i - ln(n - 1),
 * A_i = sum_{j != i} v(i, j), v(i, j) = K_h1(|x_i - x_j|) K_h2(|y_i - y_j|)
 * (h1 on x, h2 on y; the paper writes them the other way round), with the
 * radial Epanechnikov kernel of Sec. 4 or the Gaussian, normalised as the
 * oracle does.
 *
 * Dual-tree recursion (Alg. 1) over one kd-tree of the points in (x, y)
 * space: a node pair (Q, R) contributes to A_i for i in Q the sum S_R over
 * j in R, j != i.  Node pairs are either the same node or disjoint (both
 * nodes are split together), so the count of terms is n_R - [Q == R].
 *   - v_max = 0 (no pair inside the supports): the contribution is 0.
 *   - Deterministic test (Thm. 1): with v_min, v_max the kernel values at the
 *     boxes' largest and smallest distances, approximate when
 *     (n_R + 1) v_max <= (2 e^eps - 1)(n_R - 1) v_min, by the midpoint
 *     (v_max + v_min)/2 per term (Lemma 3); this guarantees |dL| <= eps.
 *   - Sampled test (Alg. 2): m pairs (i in Q, j in R, j != i) drawn
 *     uniformly, v_hat their mean, sigma the bootstrap standard deviation of
 *     the mean over B resamples; approximate by v_hat per term when
 *     z sigma / v_hat <= e^eps - 1.
 *   - Two leaves: the exact sum (base case).  Otherwise recurse on the four
 *     child pairs (a leaf stands in for its own child).
 * Random draws: SplitMix64 (Steele, Lea & Flood 2014) in counter form.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DT_LEAF 16
#define DT_PI 3.14159265358979323846

typedef struct {
    int begin, end;      /* points [begin, end) in tree order */
    int left, right;     /* children, -1 for a leaf */
    double *lo, *hi;     /* bounding box, dims + 1 coordinates (x dims, then y) */
    double acc;          /* approximated contribution per point, pushed down at the end */
} dt_node;

typedef struct {
    int n, d, D;         /* points, x dims, D = d + 1 */
    double *p;           /* points in tree order, [n][D] */
    int *perm;           /* tree position -> input index */
    dt_node *nodes;
    int n_nodes, cap;
    double *box;         /* storage of the boxes */
    int kernel;          /* 0 Gaussian, 1 Epanechnikov */
    double h1, h2, cx, cy;   /* bandwidths; log-free normalisations of K_h1 (dims d) and K_h2 (dim 1) */
    double *A;           /* per tree position */
    double eps, z;
    int mode, m, B;      /* mode 0 deterministic, 1 sampled */
    uint64_t seed, ctr;
    int64_t n_exact, n_pruned;   /* pair terms evaluated exactly / node pairs approximated */
} dt_tree;

static uint64_t dt_splitmix(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t dt_next(dt_tree* t) { return dt_splitmix(t->seed, t->ctr++); }
static int dt_below(dt_tree* t, int n) { return (int)(dt_next(t) % (uint64_t)n); }

/* unit-ball volume V_k */
static double dt_ball(int k) {
    double v = (k % 2) ? 2.0 : 1.0;
    for (int j = 2 + k % 2; j <= k; j += 2) v *= 2.0 * DT_PI / j;
    return v;
}

/* kernel profile at squared scaled distance s = r^2 / h^2 (without the constant) */
static double dt_prof(int kernel, double s) {
    if (kernel == 1) return s < 1.0 ? 1.0 - s : 0.0;
    return exp(-0.5 * s);
}

static double dt_v(const dt_tree* t, const double* a, const double* b) {
    double sx = 0.0;
    for (int c = 0; c < t->d; ++c) {
        const double q = a[c] - b[c];
        sx += q * q;
    }
    const double qy = a[t->d] - b[t->d];
    return t->cx * dt_prof(t->kernel, sx / (t->h1 * t->h1)) * t->cy * dt_prof(t->kernel, qy * qy / (t->h2 * t->h2));
}

static int dt_new_node(dt_tree* t) {
    if (t->n_nodes == t->cap) return -1;
    dt_node* nd = &t->nodes[t->n_nodes];
    nd->lo = t->box + (size_t)t->n_nodes * 2 * t->D;
    nd->hi = nd->lo + t->D;
    nd->left = nd->right = -1;
    nd->acc = 0.0;
    return t->n_nodes++;
}

static int dt_cmp_dim;
static const double* dt_cmp_p;
static int dt_cmp_D;
static int dt_cmp(const void* a, const void* b) {
    const double va = dt_cmp_p[(size_t)(*(const int*)a) * dt_cmp_D + dt_cmp_dim];
    const double vb = dt_cmp_p[(size_t)(*(const int*)b) * dt_cmp_D + dt_cmp_dim];
    return va < vb ? -1 : va > vb ? 1 : 0;
}

/* build over idx[begin, end) (indices into the input points src) */
static int dt_build(dt_tree* t, const double* src, int* idx, int begin, int end) {
    const int id = dt_new_node(t);
    if (id < 0) return -1;
    dt_node* nd = &t->nodes[id];
    nd->begin = begin;
    nd->end = end;
    for (int c = 0; c < t->D; ++c) {
        nd->lo[c] = INFINITY;
        nd->hi[c] = -INFINITY;
    }
    for (int k = begin; k < end; ++k)
        for (int c = 0; c < t->D; ++c) {
            const double v = src[(size_t)idx[k] * t->D + c];
            if (v < nd->lo[c]) nd->lo[c] = v;
            if (v > nd->hi[c]) nd->hi[c] = v;
        }
    if (end - begin <= DT_LEAF) return id;
    int wd = 0;
    for (int c = 1; c < t->D; ++c)
        if (nd->hi[c] - nd->lo[c] > nd->hi[wd] - nd->lo[wd]) wd = c;
    if (!(nd->hi[wd] > nd->lo[wd])) return id;   /* all points equal: a leaf */
    dt_cmp_dim = wd;
    dt_cmp_p = src;
    dt_cmp_D = t->D;
    qsort(idx + begin, (size_t)(end - begin), sizeof(int), dt_cmp);
    const int mid = begin + (end - begin) / 2;
    const int l = dt_build(t, src, idx, begin, mid);
    const int r = dt_build(t, src, idx, mid, end);
    if (l < 0 || r < 0) return -1;
    t->nodes[id].left = l;
    t->nodes[id].right = r;
    return id;
}

/* smallest and largest squared distance between two boxes over dims [c0, c1) */
static void dt_box_dist(const dt_node* a, const dt_node* b, int c0, int c1, double* dmin2, double* dmax2) {
    double mn = 0.0, mx = 0.0;
    for (int c = c0; c < c1; ++c) {
        double gap = a->lo[c] - b->hi[c];
        const double g2 = b->lo[c] - a->hi[c];
        if (g2 > gap) gap = g2;
        if (gap > 0.0) mn += gap * gap;
        double far = a->hi[c] - b->lo[c];
        const double f2 = b->hi[c] - a->lo[c];
        if (f2 > far) far = f2;
        mx += far * far;
    }
    *dmin2 = mn;
    *dmax2 = mx;
}

static void dt_base(dt_tree* t, const dt_node* q, const dt_node* r) {
    for (int i = q->begin; i < q->end; ++i) {
        double s = 0.0;
        for (int j = r->begin; j < r->end; ++j)
            if (j != i) s += dt_v(t, t->p + (size_t)i * t->D, t->p + (size_t)j * t->D);
        t->A[i] += s;
    }
    t->n_exact += (int64_t)(q->end - q->begin) * (r->end - r->begin);
}

/* Alg. 2: relative half-width z sigma / v_hat of the sampled mean; v_hat out */
static double dt_sample(dt_tree* t, const dt_node* q, const dt_node* r, double* vhat) {
    double s[256];
    const int m = t->m < 256 ? t->m : 256;
    const int nq = q->end - q->begin, nr = r->end - r->begin;
    for (int k = 0; k < m; ++k) {
        int i, j;
        do {
            i = q->begin + dt_below(t, nq);
            j = r->begin + dt_below(t, nr);
        } while (i == j);
        s[k] = dt_v(t, t->p + (size_t)i * t->D, t->p + (size_t)j * t->D);
    }
    double mean = 0.0;
    for (int k = 0; k < m; ++k) mean += s[k];
    mean /= m;
    *vhat = mean;
    if (!(mean > 0.0)) return INFINITY;
    double bs = 0.0, bs2 = 0.0;
    for (int b = 0; b < t->B; ++b) {
        double mb = 0.0;
        for (int k = 0; k < m; ++k) mb += s[dt_below(t, m)];
        mb /= m;
        bs += mb;
        bs2 += mb * mb;
    }
    const double bm = bs / t->B;
    double var = bs2 / t->B - bm * bm;
    if (var < 0.0) var = 0.0;
    return t->z * sqrt(var) / mean;
}

static void dt_rec(dt_tree* t, int qi, int ri) {
    dt_node* q = &t->nodes[qi];
    dt_node* r = &t->nodes[ri];
    const int nr = r->end - r->begin;
    const double cnt = (double)(nr - (qi == ri ? 1 : 0));
    double dx_mn, dx_mx, dy_mn, dy_mx;
    dt_box_dist(q, r, 0, t->d, &dx_mn, &dx_mx);
    dt_box_dist(q, r, t->d, t->D, &dy_mn, &dy_mx);
    const double vmax = t->cx * dt_prof(t->kernel, dx_mn / (t->h1 * t->h1)) *
                        t->cy * dt_prof(t->kernel, dy_mn / (t->h2 * t->h2));
    if (vmax == 0.0) {   /* no pair inside the supports */
        ++t->n_pruned;
        return;
    }
    const int both_leaves = q->left < 0 && r->left < 0;
    if (cnt >= 1.0) {
        if (t->mode == 0) {
            const double vmin = t->cx * dt_prof(t->kernel, dx_mx / (t->h1 * t->h1)) *
                                t->cy * dt_prof(t->kernel, dy_mx / (t->h2 * t->h2));
            if (nr >= 2 && vmin > 0.0 && (nr + 1) * vmax <= (2.0 * exp(t->eps) - 1.0) * (nr - 1) * vmin) {
                q->acc += cnt * 0.5 * (vmax + vmin);
                ++t->n_pruned;
                return;
            }
        } else if (!both_leaves && (int64_t)(q->end - q->begin) * nr > 2 * t->m) {
            double vhat;
            if (dt_sample(t, q, r, &vhat) <= exp(t->eps) - 1.0) {
                q->acc += cnt * vhat;
                ++t->n_pruned;
                return;
            }
        }
    }
    if (both_leaves) {
        dt_base(t, q, r);
        return;
    }
    const int ql = q->left < 0 ? qi : q->left, qr = q->left < 0 ? -1 : q->right;
    const int rl = r->left < 0 ? ri : r->left, rr = r->left < 0 ? -1 : r->right;
    if (qi == ri) {   /* the same node: its child pairs, each unordered pair once per direction */
        dt_rec(t, ql, ql);
        if (qr >= 0) {
            dt_rec(t, ql, qr);
            dt_rec(t, qr, ql);
            dt_rec(t, qr, qr);
        }
        return;
    }
    const int qs[2] = {ql, qr}, rs[2] = {rl, rr};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (qs[a] >= 0 && rs[b] >= 0) dt_rec(t, qs[a], rs[b]);
}

static void dt_push(dt_tree* t, int id, double above) {
    const dt_node* nd = &t->nodes[id];
    const double a = above + nd->acc;
    if (nd->left < 0) {
        for (int i = nd->begin; i < nd->end; ++i) t->A[i] += a;
        return;
    }
    dt_push(t, nd->left, a);
    dt_push(t, nd->right, a);
}

/*
 * The score of one bandwidth pair.  x: n x d row-major (already standardised
 * if wanted), y: n.  kernel 0 Gaussian / 1 Epanechnikov; mode 0 deterministic
 * (Thm. 1) / 1 sampled (Alg. 2, m samples, B bootstrap resamples, z).  Writes
 * L (Eq. 3; -inf when some A_i is 0) and, when the pointers are not NULL,
 * the number of pair terms evaluated exactly and of node pairs approximated.
 * Returns 0, or -1 on allocation failure or bad arguments.
 */
int dualtree_loo_eq3(const double* x, const double* y, int n, int d, double h1, double h2, int kernel,
                     int mode, double eps, int m, int B, double z, uint64_t seed, double* L,
                     int64_t* n_exact, int64_t* n_pruned) {
    if (n < 2 || d < 1 || !(h1 > 0.0) || !(h2 > 0.0) || !L) return -1;
    dt_tree t;
    memset(&t, 0, sizeof t);
    t.n = n;
    t.d = d;
    t.D = d + 1;
    t.kernel = kernel;
    t.h1 = h1;
    t.h2 = h2;
    t.eps = eps;
    t.mode = mode;
    t.m = m > 0 ? m : 25;
    t.B = B > 0 ? B : 10;
    t.z = z;
    t.seed = seed;
    /* normalisations: Gaussian (2 pi)^{-k/2} h^{-k}; Epanechnikov c_k h^{-k}, c_k = (k + 2) / (2 V_k) */
    t.cx = kernel == 1 ? (d + 2.0) / (2.0 * dt_ball(d)) * pow(h1, -d) : pow(2.0 * DT_PI, -0.5 * d) * pow(h1, -d);
    t.cy = kernel == 1 ? 3.0 / 4.0 / h2 : 1.0 / (sqrt(2.0 * DT_PI) * h2);
    double* src = (double*)malloc(sizeof(double) * (size_t)n * t.D);
    int* idx = (int*)malloc(sizeof(int) * (size_t)n);
    t.cap = 4 * (n / DT_LEAF + 1) + 8;
    t.nodes = (dt_node*)malloc(sizeof(dt_node) * (size_t)t.cap);
    t.box = (double*)malloc(sizeof(double) * (size_t)t.cap * 2 * t.D);
    t.p = (double*)malloc(sizeof(double) * (size_t)n * t.D);
    t.A = (double*)calloc((size_t)n, sizeof(double));
    int rc = -1;
    if (src && idx && t.nodes && t.box && t.p && t.A) {
        for (int i = 0; i < n; ++i) {
            for (int c = 0; c < d; ++c) src[(size_t)i * t.D + c] = x[(size_t)i * d + c];
            src[(size_t)i * t.D + d] = y[i];
            idx[i] = i;
        }
        if (dt_build(&t, src, idx, 0, n) == 0) {
            for (int k = 0; k < n; ++k) memcpy(t.p + (size_t)k * t.D, src + (size_t)idx[k] * t.D, sizeof(double) * t.D);
            dt_rec(&t, 0, 0);
            dt_push(&t, 0, 0.0);
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += log(t.A[i]);   /* -inf when an A_i is 0 */
            *L = s / n - log(n - 1.0);
            if (n_exact) *n_exact = t.n_exact;
            if (n_pruned) *n_pruned = t.n_pruned;
            rc = 0;
        }
    }
    free(src);
    free(idx);
    free(t.nodes);
    free(t.box);
    free(t.p);
    free(t.A);
    return rc;
}
