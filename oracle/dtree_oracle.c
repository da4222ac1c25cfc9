/*
 * dtree_oracle.c -- CPU reference ("oracle") for exact k-nearest-neighbour search.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the package's smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * Everything is plain, serial-per-query C in IEEE double precision, compiled
 * with -ffp-contract=off so that every squared distance is the same bit
 * pattern on every host:
 *
 *     d2(q, r) = sum_{j = 0 .. d-1} (double(q_j) - double(r_j))^2,
 *
 * summed left to right with one rounding per operation.
 *
 * Source: Curtin, March, Ram, Anderson, Gray, Isbell, "Tree-Independent
 * Dual-Tree Algorithms", ICML 2013.
 *   - kNN problem statement, Section 5: queries S_q (n x d), references S_r
 *     (m x d), 0 < k < m; N_p / D_p ordered nearest-first; D_p[i] = inf past
 *     the end of the list; in the monochromatic case a point does not return
 *     itself (footnote to Algorithm 2).
 *   - Space tree (Definition 1) and the quantities d_min, rho, lambda
 *     (Section 3 definitions) with the kd-tree bounds given after them.
 *   - DepthFirstTraversal (Algorithm 1), kNN BaseCase (Algorithm 2),
 *     kNN Score (Algorithm 3), the bounds B_1, B_2 and the combined B
 *     (Section 5), Gray's AllNN (Algorithm 4).
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *   R1  Euclidean metric; lists compared on squared distance.
 *   R2  ties in distance are broken by the lower reference index, so
 *       "(d2, index) lexicographically smaller" replaces "d < D[k]".
 *   R3  a node pair is pruned only when d_min > B (strictly), so an equal
 *       distance, lower index candidate is never lost.
 *   R4  the combined bound is evaluated in its sound form
 *         B(N) = min over N and its ancestors a of min(B_1(a), A(a) + 2 lambda(a)),
 *       A(a) = min over descendant points of D_p[k].  The recursion exactly
 *       as printed in Section 5 is kept as variant BOUND_LITERAL.
 *   R5  max over an empty set = -inf, min over an empty set = +inf; kd-tree
 *       internal nodes hold no points, leaves hold all of theirs, so
 *       rho(leaf) = lambda(leaf).
 *   R6  the centroid C of a node is the centre of its bounding box; lambda is
 *       the exact maximum over descendant points.
 *   R7  the node's convex set is the tight bounding box of its points.
 *   R8  in Algorithm 1 a childless node stands in for itself and recursion
 *       stops when both nodes are leaves.
 *   R9  monochromatic self-exclusion is by index, not by zero distance.
 *   R11 kd construction: split on the widest box dimension (lower dimension
 *       on ties) at the index median, left child = floor(n/2) smallest by
 *       (coordinate, index); a node with n <= leaf_size is a leaf.
 *   R12 in Algorithm 4 the leaf-level bound is delta = max over the leaf's
 *       points of D_p (the text says delta equals B_1); the printed
 *       per-pair line "if d < delta then delta = d" is kept as a variant.
 *   R13 Score's d_min may be any lower bound on the distance between the two
 *       nodes' points (Section 3 asks a space tree only for d_min, rho and
 *       lambda): the boxes' distance (the kd-tree), the distance between the
 *       balls of radius lambda around the box centres (a ball tree over the
 *       same splits: by R6 every point of a node lies within lambda of its
 *       centre), or the larger of the two.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

enum {
    BOUND_SOUND = 0,    /* R4 */
    BOUND_LITERAL = 1,  /* the printed recursion of Section 5, unchanged */
    BOUND_B1 = 2,       /* B_1 alone (Gray's delta) */
    BOUND_NONE = 3      /* never prune: the plain dual-tree traversal */
};

enum {
    DMIN_BOX = 0,   /* R13: the boxes */
    DMIN_BALL = 1,  /* R13: the balls */
    DMIN_BOTH = 2   /* R13: the larger of the two */
};

/* stats[] slots filled by oracle_knn_dualtree */
enum {
    ST_SCORES = 0,       /* Score() calls */
    ST_PRUNES = 1,       /* pairs pruned */
    ST_LEAF_PAIRS = 2,   /* leaf x leaf pairs whose BaseCase loop ran */
    ST_BASECASES = 3,    /* BaseCase(p_q, p_r) calls */
    ST_AUDIT_PRUNE = 4,  /* pruned pairs whose reference node held a true neighbour */
    ST_AUDIT_BOUND = 5,  /* Score calls where B(N_q) < max true D_p[k] over D^p_q */
    ST_ORDER = 6,        /* Score calls where B(N_q) > B_1(N_q) or B(N_q) > B(Par(N_q)) */
    ST_QNODES = 7,       /* nodes in the query tree */
    ST_INCOMPLETE = 8,   /* queries left with fewer than k neighbours (unsound bound) */
    ST_NSTATS = 9
};

static const double INF = 1.0 / 0.0;

/* ---------------------------------------------------------------------- */
/* distance: the definition of the problem                                 */
/* ---------------------------------------------------------------------- */

static double sqdist(const float* a, const float* b, int d) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = (double)a[j] - (double)b[j];
        s += t * t;
    }
    return s;
}

/* (d2a, ia) < (d2b, ib) lexicographically (R2) */
static int key_less(double d2a, int64_t ia, double d2b, int64_t ib) {
    if (d2a < d2b) return 1;
    if (d2a > d2b) return 0;
    return ia < ib;
}

/* Insert (d2, idx) into the list of length k kept ascending by (d2, idx);
 * the last entry falls off.  Returns 1 if inserted.  Empty slots hold
 * (+inf, -1), which every real candidate beats (D_p[i] = inf past the end). */
static int list_insert(double* D2, int64_t* N, int k, double d2, int64_t idx) {
    if (!(N[k - 1] < 0 || key_less(d2, idx, D2[k - 1], N[k - 1]))) return 0;
    for (int i = 0; i < k; ++i)
        if (N[i] == idx) return 0;           /* "BaseCase not yet called" guard */
    int pos = k - 1;
    while (pos > 0 && (N[pos - 1] < 0 || key_less(d2, idx, D2[pos - 1], N[pos - 1]))) {
        D2[pos] = D2[pos - 1];
        N[pos] = N[pos - 1];
        --pos;
    }
    D2[pos] = d2;
    N[pos] = idx;
    return 1;
}

/* ---------------------------------------------------------------------- */
/* brute force: compare every pair, keep the k smallest (Section 5)        */
/* ---------------------------------------------------------------------- */

/* q: nq x d, r: nr x d, row-major float32.  self_idx (nullable): reference
 * index that query i must not return (monochromatic case, R9), or -1.
 * out_idx / out_d2: nq x k, ascending by (d2, index). */
int oracle_knn_brute(const float* q, int64_t nq, const float* r, int64_t nr, int32_t d,
                     int32_t k, const int64_t* self_idx, int64_t* out_idx, double* out_d2) {
    if (!q || !r || !out_idx || !out_d2 || d <= 0 || k <= 0 || nq < 0 || nr <= 0)
        return ORACLE_EINVAL;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : bad)
    for (int64_t i = 0; i < nq; ++i) {
        double* D2 = out_d2 + i * k;
        int64_t* N = out_idx + i * k;
        for (int j = 0; j < k; ++j) { D2[j] = INF; N[j] = -1; }
        const float* qi = q + i * (int64_t)d;
        int64_t skip = self_idx ? self_idx[i] : -1;
        for (int64_t j = 0; j < nr; ++j) {
            if (j == skip) continue;
            double d2 = sqdist(qi, r + j * (int64_t)d, d);
            if (N[k - 1] < 0 || key_less(d2, j, D2[k - 1], N[k - 1])) {
                int pos = k - 1;
                while (pos > 0 && (N[pos - 1] < 0 || key_less(d2, j, D2[pos - 1], N[pos - 1]))) {
                    D2[pos] = D2[pos - 1];
                    N[pos] = N[pos - 1];
                    --pos;
                }
                D2[pos] = d2;
                N[pos] = j;
            }
        }
        if (N[k - 1] < 0) bad = 1;   /* fewer than k candidates: k too large */
    }
    return bad ? ORACLE_EINVAL : ORACLE_OK;
}

/* ---------------------------------------------------------------------- */
/* kd-tree (a space tree, Definition 1; construction R11)                  */
/* ---------------------------------------------------------------------- */

typedef struct {
    int d, leaf;
    int64_t n;
    const float* pts;
    int64_t* perm;      /* tree position -> original row */
    int64_t* iperm;     /* original row -> tree position */
    int32_t nnodes, cap;
    int64_t *begin, *count;
    int32_t *left, *right, *parent;
    double *lo, *hi;    /* nnodes x d, tight bounding box (R7) */
    double* lambda;     /* max distance from box centre to descendant points (R6) */
} otree;

typedef struct { const float* pts; int d; int dim; } sortctx;

static int perm_less(const sortctx* c, int64_t a, int64_t b) {
    float va = c->pts[a * c->d + c->dim], vb = c->pts[b * c->d + c->dim];
    if (va < vb) return 1;
    if (va > vb) return 0;
    return a < b;
}

static void merge_sort(const sortctx* c, int64_t* a, int64_t* tmp, int64_t n) {
    if (n < 2) return;
    int64_t h = n / 2;
    merge_sort(c, a, tmp, h);
    merge_sort(c, a + h, tmp, n - h);
    int64_t i = 0, j = h, o = 0;
    while (i < h && j < n) tmp[o++] = perm_less(c, a[j], a[i]) ? a[j++] : a[i++];
    while (i < h) tmp[o++] = a[i++];
    while (j < n) tmp[o++] = a[j++];
    memcpy(a, tmp, (size_t)n * sizeof(int64_t));
}

static int tree_grow(otree* t) {
    int32_t cap = t->cap ? t->cap * 2 : 64;
    int d = t->d;
#define GROW(p, T, m)                                                         \
    do {                                                                      \
        T* np_ = (T*)realloc(t->p, (size_t)cap * (m) * sizeof(T));            \
        if (!np_) return ORACLE_ENOMEM;                                       \
        t->p = np_;                                                           \
    } while (0)
    GROW(begin, int64_t, 1); GROW(count, int64_t, 1);
    GROW(left, int32_t, 1); GROW(right, int32_t, 1); GROW(parent, int32_t, 1);
    GROW(lo, double, d); GROW(hi, double, d); GROW(lambda, double, 1);
#undef GROW
    t->cap = cap;
    return ORACLE_OK;
}

static int32_t build_node(otree* t, int64_t* tmp, int64_t b, int64_t n, int32_t par, int* err) {
    if (*err) return -1;
    if (t->nnodes == t->cap && (*err = tree_grow(t))) return -1;
    int32_t id = t->nnodes++;
    int d = t->d;
    t->begin[id] = b; t->count[id] = n; t->parent[id] = par;
    t->left[id] = t->right[id] = -1;
    double* lo = t->lo + (int64_t)id * d;
    double* hi = t->hi + (int64_t)id * d;
    for (int j = 0; j < d; ++j) { lo[j] = INF; hi[j] = -INF; }
    for (int64_t i = b; i < b + n; ++i) {
        const float* p = t->pts + t->perm[i] * d;
        for (int j = 0; j < d; ++j) {
            if (p[j] < lo[j]) lo[j] = p[j];
            if (p[j] > hi[j]) hi[j] = p[j];
        }
    }
    double lam = 0.0;                      /* exact lambda, centroid = box centre */
    for (int64_t i = b; i < b + n; ++i) {
        const float* p = t->pts + t->perm[i] * d;
        double s = 0.0;
        for (int j = 0; j < d; ++j) {
            double c = 0.5 * (lo[j] + hi[j]);
            double u = c - (double)p[j];
            s += u * u;
        }
        if (sqrt(s) > lam) lam = sqrt(s);
    }
    t->lambda[id] = lam;
    if (n <= t->leaf) return id;
    int dim = 0;
    for (int j = 1; j < d; ++j)
        if (hi[j] - lo[j] > hi[dim] - lo[dim]) dim = j;
    sortctx c = {t->pts, d, dim};
    merge_sort(&c, t->perm + b, tmp, n);
    int64_t nl = n / 2;
    int32_t l = build_node(t, tmp, b, nl, id, err);
    int32_t r = build_node(t, tmp, b + nl, n - nl, id, err);
    t->left[id] = l;
    t->right[id] = r;
    return id;
}

static void tree_free(otree* t) {
    free(t->perm); free(t->iperm); free(t->begin); free(t->count);
    free(t->left); free(t->right); free(t->parent);
    free(t->lo); free(t->hi); free(t->lambda);
    memset(t, 0, sizeof(*t));
}

static int tree_build(otree* t, const float* pts, int64_t n, int d, int leaf) {
    memset(t, 0, sizeof(*t));
    t->pts = pts; t->n = n; t->d = d; t->leaf = leaf;
    t->perm = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    t->iperm = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* tmp = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!t->perm || !t->iperm || !tmp) { free(tmp); tree_free(t); return ORACLE_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) t->perm[i] = i;
    int err = 0;
    build_node(t, tmp, 0, n, -1, &err);
    free(tmp);
    if (err) { tree_free(t); return err; }
    for (int64_t i = 0; i < n; ++i) t->iperm[t->perm[i]] = i;
    return ORACLE_OK;
}

static int is_leaf(const otree* t, int32_t id) { return t->left[id] < 0; }

/* d_min between two nodes, bounded below by the distance between their
 * boxes (kd-tree bound after the Section 3 definitions). */
static double box_dmin(const otree* tq, int32_t a, const otree* tr, int32_t b) {
    int d = tq->d;
    const double *lq = tq->lo + (int64_t)a * d, *hq = tq->hi + (int64_t)a * d;
    const double *lr = tr->lo + (int64_t)b * d, *hr = tr->hi + (int64_t)b * d;
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double g = 0.0;
        if (lq[j] > hr[j]) g = lq[j] - hr[j];
        else if (lr[j] > hq[j]) g = lr[j] - hq[j];
        s += g * g;
    }
    return sqrt(s);
}

/* ---------------------------------------------------------------------- */
/* dual-tree kNN: Algorithm 1 + Algorithm 2 + Algorithm 3                  */
/* ---------------------------------------------------------------------- */

typedef struct {
    const otree *tq, *tr;
    int k, mono, bound_kind, dmin_kind;
    int32_t stop;              /* the bound's ancestor chain ends at this node */
    double* D2;                /* nq x k, indexed by original query row */
    int64_t* N;
    double *B1, *A, *Blit;     /* per query node caches (distance units) */
    const int64_t* true_idx;   /* audit: brute-force lists (nullable) */
    const double* true_maxdk;  /* audit: per query node max true D_p[k] */
    int64_t st[ST_NSTATS];
} kctx;

/* d_min between the balls around the box centres of radius lambda (R13):
 * |C_a - C_b| - lambda_a - lambda_b, or 0 when the balls meet. */
static double ball_dmin(const otree* tq, int32_t a, const otree* tr, int32_t b) {
    int d = tq->d;
    const double *lq = tq->lo + (int64_t)a * d, *hq = tq->hi + (int64_t)a * d;
    const double *lr = tr->lo + (int64_t)b * d, *hr = tr->hi + (int64_t)b * d;
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = 0.5 * (lq[j] + hq[j]) - 0.5 * (lr[j] + hr[j]);
        s += t * t;
    }
    double g = sqrt(s) - tq->lambda[a] - tr->lambda[b];
    return g > 0.0 ? g : 0.0;
}

/* Score's d_min under the traversal's choice (R13). */
static double node_dmin(const kctx* c, int32_t a, int32_t b) {
    switch (c->dmin_kind) {
    case DMIN_BALL: return ball_dmin(c->tq, a, c->tr, b);
    case DMIN_BOTH: return fmax(box_dmin(c->tq, a, c->tr, b), ball_dmin(c->tq, a, c->tr, b));
    default: return box_dmin(c->tq, a, c->tr, b);
    }
}

static double kth(const kctx* c, int64_t q) {
    return c->N[q * c->k + c->k - 1] < 0 ? INF : sqrt(c->D2[q * c->k + c->k - 1]);
}

static double bound_of(const kctx* c, int32_t n) {
    const otree* t = c->tq;
    double b = INF;
    switch (c->bound_kind) {
    case BOUND_NONE:
        return INF;
    case BOUND_B1:
        return c->B1[n];
    case BOUND_LITERAL:
        for (int32_t a = n; a >= 0; a = (a == c->stop) ? -1 : t->parent[a])
            if (c->Blit[a] < b) b = c->Blit[a];
        return b;
    default:
        for (int32_t a = n; a >= 0; a = (a == c->stop) ? -1 : t->parent[a]) {
            double b2 = c->A[a] + 2.0 * t->lambda[a];
            if (c->B1[a] < b) b = c->B1[a];
            if (b2 < b) b = b2;
        }
        return b;
    }
}

/* Recompute the cached B_1, A (and the literal recursion) of leaf n from its
 * points, then of every ancestor from its children. */
static void refresh_bounds(kctx* c, int32_t n) {
    const otree* t = c->tq;
    double b1 = -INF, a = INF;
    for (int64_t i = t->begin[n]; i < t->begin[n] + t->count[n]; ++i) {
        double v = kth(c, t->perm[i]);
        if (v > b1) b1 = v;
        if (v < a) a = v;
    }
    c->B1[n] = b1;
    c->A[n] = a;
    c->Blit[n] = fmin(b1, a + 2.0 * t->lambda[n]);      /* terms 1 and 2, leaf (R5) */
    /* the walk ends at this context's own subtree root: a leaf that is the
     * root itself has no ancestor of its own to refresh */
    for (int32_t p = (n == c->stop) ? -1 : t->parent[n]; p >= 0; p = t->parent[p]) {
        int32_t l = t->left[p], r = t->right[p];
        c->B1[p] = fmax(c->B1[l], c->B1[r]);
        c->A[p] = fmin(c->A[l], c->A[r]);
        /* printed recursion: min{ max{max_P D, max_c B(c)}, min_P(D+rho+lambda),
         * min_c(B(c) + 2(lambda - lambda_c)) }, with P empty for internal nodes */
        double t1 = fmax(c->Blit[l], c->Blit[r]);
        double t3 = fmin(c->Blit[l] + 2.0 * (t->lambda[p] - t->lambda[l]),
                         c->Blit[r] + 2.0 * (t->lambda[p] - t->lambda[r]));
        c->Blit[p] = fmin(t1, t3);
        if (p == c->stop) break;
    }
}

static void base_case_leaves(kctx* c, int32_t nq, int32_t nr) {
    const otree *tq = c->tq, *tr = c->tr;
    int d = tq->d, k = c->k;
    c->st[ST_LEAF_PAIRS]++;
    for (int64_t i = tq->begin[nq]; i < tq->begin[nq] + tq->count[nq]; ++i) {
        int64_t pq = tq->perm[i];
        for (int64_t j = tr->begin[nr]; j < tr->begin[nr] + tr->count[nr]; ++j) {
            int64_t pr = tr->perm[j];
            if (c->mono && pq == pr) continue;                   /* R9 */
            c->st[ST_BASECASES]++;
            double d2 = sqdist(tq->pts + pq * d, tr->pts + pr * d, d);
            list_insert(c->D2 + pq * k, c->N + pq * k, k, d2, pr);
        }
    }
    refresh_bounds(c, nq);
}

static void audit_prune(kctx* c, int32_t nq, int32_t nr) {
    const otree *tq = c->tq, *tr = c->tr;
    int k = c->k;
    int64_t rb = tr->begin[nr], re = rb + tr->count[nr];
    for (int64_t i = tq->begin[nq]; i < tq->begin[nq] + tq->count[nq]; ++i) {
        int64_t pq = tq->perm[i];
        for (int j = 0; j < k; ++j) {
            int64_t pos = tr->iperm[c->true_idx[pq * k + j]];
            if (pos >= rb && pos < re) { c->st[ST_AUDIT_PRUNE]++; return; }
        }
    }
}

static void traverse(kctx* c, int32_t nq, int32_t nr) {
    const otree *tq = c->tq, *tr = c->tr;
    c->st[ST_SCORES]++;
    double B = bound_of(c, nq);
    if (c->true_maxdk && B < c->true_maxdk[nq] * (1.0 - 1e-12)) c->st[ST_AUDIT_BOUND]++;
    if (c->bound_kind == BOUND_SOUND) {
        if (B > c->B1[nq]) c->st[ST_ORDER]++;
        if (nq != c->stop && tq->parent[nq] >= 0 && B > bound_of(c, tq->parent[nq]))
            c->st[ST_ORDER]++;
    }
    double dmin = node_dmin(c, nq, nr);
    if (dmin > B) {                                              /* Score = inf (R3) */
        c->st[ST_PRUNES]++;
        if (c->true_idx) audit_prune(c, nq, nr);
        return;
    }
    int lq = is_leaf(tq, nq), lr = is_leaf(tr, nr);
    if (lq && lr) { base_case_leaves(c, nq, nr); return; }      /* R8 */
    int32_t qs[2] = {lq ? nq : tq->left[nq], lq ? -1 : tq->right[nq]};
    for (int a = 0; a < 2 && qs[a] >= 0; ++a) {
        int32_t qc = qs[a];
        if (lr) { traverse(c, qc, nr); continue; }
        int32_t r0 = tr->left[nr], r1 = tr->right[nr];
        if (node_dmin(c, qc, r1) < node_dmin(c, qc, r0)) {        /* closer first */
            int32_t s = r0; r0 = r1; r1 = s;
        }
        traverse(c, qc, r0);
        traverse(c, qc, r1);
    }
}

static void true_max_dk(const otree* t, int32_t n, const double* true_d2, int k, double* out) {
    if (is_leaf(t, n)) {
        double m = -INF;
        for (int64_t i = t->begin[n]; i < t->begin[n] + t->count[n]; ++i) {
            double v = sqrt(true_d2[t->perm[i] * k + k - 1]);
            if (v > m) m = v;
        }
        out[n] = m;
        return;
    }
    true_max_dk(t, t->left[n], true_d2, k, out);
    true_max_dk(t, t->right[n], true_d2, k, out);
    out[n] = fmax(out[t->left[n]], out[t->right[n]]);
}

/* Dual-tree exact kNN.
 *   q == NULL (or mono != 0): monochromatic, the reference tree is also the
 *     query tree and a point never returns itself (R9).
 *   bound_kind: BOUND_SOUND / BOUND_LITERAL / BOUND_B1 / BOUND_NONE.
 *   dmin_kind: DMIN_BOX / DMIN_BALL / DMIN_BOTH, Score's d_min (R13).
 *   par_depth: 0 runs Algorithm 1 once from the two roots.  p > 0 runs one
 *     independent traversal per query node at depth p (in parallel), each
 *     from that node and the reference root, and ends the bound's ancestor
 *     chain at that node.
 *   true_idx / true_d2 (nullable): brute-force lists, enabling the audit
 *     counters ST_AUDIT_PRUNE and ST_AUDIT_BOUND.
 *   stats (nullable): ST_NSTATS counters.  A query left with fewer than k
 *     neighbours (possible only with an unsound bound) keeps -1 / +inf slots
 *     and is counted in ST_INCOMPLETE.
 * Output: out_idx / out_d2 (nq x k) ascending by (d2, index). */
int oracle_knn_dualtree(const float* q, int64_t nq, const float* r, int64_t nr, int32_t d,
                        int32_t k, int32_t mono, int32_t leaf_size, int32_t bound_kind,
                        int32_t dmin_kind, int32_t par_depth, const int64_t* true_idx,
                        const double* true_d2, int64_t* out_idx, double* out_d2, int64_t* stats) {
    if (!r || !out_idx || !out_d2 || d <= 0 || k <= 0 || nr <= 0 || leaf_size < 1 ||
        bound_kind < 0 || bound_kind > 3 || dmin_kind < 0 || dmin_kind > 2 || par_depth < 0)
        return ORACLE_EINVAL;
    mono = mono || q == NULL;
    if (mono) { q = r; nq = nr; }
    if (k > (mono ? nr - 1 : nr)) return ORACLE_EINVAL;
    otree tr, tq_own;
    int rc = tree_build(&tr, r, nr, d, leaf_size);
    if (rc) return rc;
    const otree* tq = &tr;
    if (!mono) {
        if ((rc = tree_build(&tq_own, q, nq, d, leaf_size))) { tree_free(&tr); return rc; }
        tq = &tq_own;
    }
    int32_t nn = tq->nnodes;
    double* B1 = (double*)malloc((size_t)nn * sizeof(double));
    double* A = (double*)malloc((size_t)nn * sizeof(double));
    double* Bl = (double*)malloc((size_t)nn * sizeof(double));
    double* tmax = true_d2 ? (double*)malloc((size_t)nn * sizeof(double)) : NULL;
    if (!B1 || !A || !Bl || (true_d2 && !tmax)) { rc = ORACLE_ENOMEM; goto done; }
    for (int32_t i = 0; i < nn; ++i) { B1[i] = INF; A[i] = INF; Bl[i] = INF; }
    for (int64_t i = 0; i < nq * k; ++i) { out_d2[i] = INF; out_idx[i] = -1; }
    if (tmax) true_max_dk(tq, 0, true_d2, k, tmax);

    /* roots of the independent traversals */
    int32_t* roots = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
    int32_t* depth = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
    if (!roots || !depth) { free(roots); free(depth); rc = ORACLE_ENOMEM; goto done; }
    int32_t nroots = 0;
    for (int32_t i = 0; i < nn; ++i) {
        depth[i] = tq->parent[i] < 0 ? 0 : depth[tq->parent[i]] + 1;   /* preorder ids */
        if (depth[i] == par_depth || (depth[i] < par_depth && is_leaf(tq, i))) roots[nroots++] = i;
    }
    int64_t tot[ST_NSTATS] = {0};
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t s = 0; s < nroots; ++s) {
        kctx c;
        memset(&c, 0, sizeof(c));
        c.tq = tq; c.tr = &tr; c.k = k; c.mono = mono; c.bound_kind = bound_kind;
        c.dmin_kind = dmin_kind;
        c.stop = roots[s];
        c.D2 = out_d2; c.N = out_idx; c.B1 = B1; c.A = A; c.Blit = Bl;
        c.true_idx = true_idx; c.true_maxdk = tmax;
        traverse(&c, roots[s], 0);
#pragma omp critical
        for (int j = 0; j < ST_NSTATS; ++j) tot[j] += c.st[j];
    }
    tot[ST_QNODES] = nn;
    for (int64_t i = 0; i < nq; ++i)
        if (out_idx[i * k + k - 1] < 0) tot[ST_INCOMPLETE]++;
    if (stats) memcpy(stats, tot, sizeof(tot));
    free(roots);
    free(depth);
done:
    free(B1); free(A); free(Bl); free(tmax);
    tree_free(&tr);
    if (!mono) tree_free(&tq_own);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Gray's all-nearest-neighbours, k = 1 (Algorithm 4)                      */
/* ---------------------------------------------------------------------- */

typedef struct {
    const otree *tq, *tr;
    int mono, variant;
    double* D2;        /* nearest squared distance per query row */
    int64_t* N;
    double* delta;     /* per query node bound, in distance units */
} gctx;

static void allnn(gctx* c, int32_t nq, int32_t nr) {
    const otree *tq = c->tq, *tr = c->tr;
    int d = tq->d;
    if (box_dmin(tq, nq, tr, nr) > c->delta[nq]) return;            /* R3 */
    int lq = is_leaf(tq, nq), lr = is_leaf(tr, nr);
    if (lq && lr) {
        double dmax = -INF;
        for (int64_t i = tq->begin[nq]; i < tq->begin[nq] + tq->count[nq]; ++i) {
            int64_t pq = tq->perm[i];
            for (int64_t j = tr->begin[nr]; j < tr->begin[nr] + tr->count[nr]; ++j) {
                int64_t pr = tr->perm[j];
                if (c->mono && pq == pr) continue;
                double d2 = sqdist(tq->pts + pq * d, tr->pts + pr * d, d);
                if (c->N[pq] < 0 || key_less(d2, pr, c->D2[pq], c->N[pq])) {
                    c->D2[pq] = d2;
                    c->N[pq] = pr;
                }
                if (c->variant == 1 && sqrt(d2) < c->delta[nq]) c->delta[nq] = sqrt(d2);
            }
            double dq = c->N[pq] < 0 ? INF : sqrt(c->D2[pq]);
            if (dq > dmax) dmax = dq;
        }
        if (c->variant == 0) c->delta[nq] = dmax;                         /* R12 */
        return;
    }
    int32_t qs[2] = {lq ? nq : tq->left[nq], lq ? -1 : tq->right[nq]};
    for (int a = 0; a < 2 && qs[a] >= 0; ++a) {
        int32_t qc = qs[a];
        if (lr) { allnn(c, qc, nr); continue; }
        int32_t r0 = tr->left[nr], r1 = tr->right[nr];
        if (box_dmin(tq, qc, tr, r1) < box_dmin(tq, qc, tr, r0)) { int32_t s = r0; r0 = r1; r1 = s; }
        allnn(c, qc, r0);
        allnn(c, qc, r1);
    }
    if (!lq) {
        double m = fmax(c->delta[tq->left[nq]], c->delta[tq->right[nq]]);
        if (m < c->delta[nq]) c->delta[nq] = m;
    }
}

/* variant 0: reading R12 (leaf delta = max D_p); 1: the printed per-pair line. */
int oracle_allnn_gray(const float* q, int64_t nq, const float* r, int64_t nr, int32_t d,
                      int32_t mono, int32_t leaf_size, int32_t variant, int64_t* out_idx,
                      double* out_d2) {
    if (!r || !out_idx || !out_d2 || d <= 0 || nr <= 0 || leaf_size < 1) return ORACLE_EINVAL;
    mono = mono || q == NULL;
    if (mono) { q = r; nq = nr; }
    if (nr < (mono ? 2 : 1)) return ORACLE_EINVAL;
    otree tr, tq_own;
    int rc = tree_build(&tr, r, nr, d, leaf_size);
    if (rc) return rc;
    const otree* tq = &tr;
    if (!mono) {
        if ((rc = tree_build(&tq_own, q, nq, d, leaf_size))) { tree_free(&tr); return rc; }
        tq = &tq_own;
    }
    double* delta = (double*)malloc((size_t)tq->nnodes * sizeof(double));
    if (!delta) { rc = ORACLE_ENOMEM; goto done; }
    for (int32_t i = 0; i < tq->nnodes; ++i) delta[i] = INF;
    for (int64_t i = 0; i < nq; ++i) { out_d2[i] = INF; out_idx[i] = -1; }
    gctx c = {tq, &tr, mono, variant, out_d2, out_idx, delta};
    allnn(&c, 0, 0);
    free(delta);
done:
    tree_free(&tr);
    if (!mono) tree_free(&tq_own);
    return rc;
}

/* Tree summary for tests: node count, leaf count, max depth, and whether
 * every box contains its children's boxes and every point of the node. */
int oracle_kdtree_check(const float* pts, int64_t n, int32_t d, int32_t leaf_size, int64_t* out4) {
    otree t;
    int rc = tree_build(&t, pts, n, d, leaf_size);
    if (rc) return rc;
    int64_t leaves = 0, maxdepth = 0, bad = 0;
    int32_t* depth = (int32_t*)calloc((size_t)t.nnodes, sizeof(int32_t));
    for (int32_t i = 0; i < t.nnodes; ++i) {
        if (t.parent[i] >= 0) depth[i] = depth[t.parent[i]] + 1;
        if (depth[i] > maxdepth) maxdepth = depth[i];
        if (is_leaf(&t, i)) { leaves++; if (t.count[i] > leaf_size) bad++; }
        else if (t.count[t.left[i]] != t.count[i] / 2) bad++;
        for (int64_t p = t.begin[i]; p < t.begin[i] + t.count[i]; ++p)
            for (int j = 0; j < d; ++j) {
                float v = pts[t.perm[p] * d + j];
                if (v < t.lo[(int64_t)i * d + j] || v > t.hi[(int64_t)i * d + j]) bad++;
            }
        if (t.parent[i] >= 0)
            for (int j = 0; j < d; ++j)
                if (t.lo[(int64_t)i * d + j] < t.lo[(int64_t)t.parent[i] * d + j] ||
                    t.hi[(int64_t)i * d + j] > t.hi[(int64_t)t.parent[i] * d + j]) bad++;
    }
    out4[0] = t.nnodes; out4[1] = leaves; out4[2] = maxdepth; out4[3] = bad;
    free(depth);
    tree_free(&t);
    return ORACLE_OK;
}

/* Threads used by the OpenMP loops (<= 0: leave the runtime default). */
int oracle_set_threads(int32_t n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
