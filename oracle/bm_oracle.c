/*
 * bm_oracle.c -- plain, slow CPU oracle for exact Ball Mapper construction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Every routine follows a definition of the paper literally, in FP64:
 *   - squared distance  D(a,b) = sum_i (a_i - b_i)^2, summed in index order
 *     (Euclidean metric, Sec. 2.1 and Sec. 6.1);
 *   - open ball / exact range set  R_r(q) = { x : d(q,x) < r }
 *     (Sec. 2.1, ball definition; Sec. 5, Def. 5.1 of the exact range set),
 *     evaluated as D(q,x) < r^2 by a full scan over all points;
 *   - greedy epsilon-net (Sec. 2.2 procedure): while a point is uncovered,
 *     select one (the smallest uncovered index), add it to the landmark set
 *     and mark every point of its open ball covered;
 *   - ball membership X_i = X intersect B(l_i, eps), the full ball (Sec. 2.3);
 *   - nerve 1-skeleton (Sec. 2.1 nerve definition, Sec. 5.2, Def. 5.6 of N_r(L)):
 *     edge {i,j} iff the two membership lists intersect;
 *   - target-occupancy scale (Sec. 6.1): distance of each point to its k-th
 *     nearest neighbour, the point itself counted first;
 *   - ball tree construction and range query (Sec. 3.1), an independent
 *     exact range oracle used to cross-check the brute force one;
 *   - farthest point sampling (Sec. 2.2, the deterministic alternative to the
 *     greedy): start from a given landmark, repeatedly take the point farthest
 *     from the landmark set while that distance is at least eps;
 *   - coloring (Sec. 2.3): a statistic of a per-point function f over every
 *     ball X_i (mean, median, minimum, maximum);
 *   - a graph-based conservative range oracle (Sec. 5.4, the proximity-graph
 *     family of non-exhaustive indexes): a query examines only the points its
 *     traversal of a proximity graph visits and decides membership exactly.
 *
 * Parallelism: outer loops whose iterations are independent (one query row,
 * one landmark pair row, one k-NN row) run under OpenMP.  This does not
 * change any arithmetic: each value is still computed by the same sequential
 * FP64 sum.  Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* D(a,b) = sum_{i<d} (a_i - b_i)^2 in FP64, index order. */
static double sqdist(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = a[i] - b[i];
        s += t * t;
    }
    return s;
}

int bmo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void bmo_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ---------------------------------------------------------------------------
 * Greedy epsilon-net, Sec. 2.2.  The selection rule "select an uncovered
 * point" is read as: the smallest uncovered index.  Marking covers the open
 * ball: D(x, y) < eps2.  Returns the landmark count; landmarks[] receives the
 * landmark ids in selection order (hence strictly increasing).
 * ------------------------------------------------------------------------- */
int64_t bmo_greedy(const double* X, int64_t n, int d, double eps2, int32_t* landmarks) {
    unsigned char* covered = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!covered) return -1;
    int64_t L = 0;
    for (int64_t x = 0; x < n; ++x) {
        if (covered[x]) continue;
        landmarks[L++] = (int32_t)x;
        const double* px = X + (size_t)x * d;
        #pragma omp parallel for schedule(static)
        for (int64_t y = 0; y < n; ++y) {
            if (sqdist(px, X + (size_t)y * d, d) < eps2) covered[y] = 1;
        }
    }
    free(covered);
    return L;
}

/* ---------------------------------------------------------------------------
 * Exact range oracle R_r(q) by full scan (Sec. 5, Def. 5.1), two phases.
 * counts[j] = |{ i : D(X_i, Q_j) < eps2 }|.
 * ------------------------------------------------------------------------- */
void bmo_range_count(const double* X, int64_t n, int d, const double* Q, int64_t m,
                     double eps2, int64_t* counts) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < m; ++j) {
        const double* q = Q + (size_t)j * d;
        int64_t c = 0;
        for (int64_t i = 0; i < n; ++i)
            if (sqdist(q, X + (size_t)i * d, d) < eps2) ++c;
        counts[j] = c;
    }
}

/* ids[offsets[j] ..] = the members of R(Q_j) in ascending index order. */
void bmo_range_fill(const double* X, int64_t n, int d, const double* Q, int64_t m,
                    double eps2, const int64_t* offsets, int32_t* ids) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < m; ++j) {
        const double* q = Q + (size_t)j * d;
        int64_t o = offsets[j];
        for (int64_t i = 0; i < n; ++i)
            if (sqdist(q, X + (size_t)i * d, d) < eps2) ids[o++] = (int32_t)i;
    }
}

/* Exact squared distances for listed (row, col) pairs: out[k] = D(Q_row, X_col). */
void bmo_pair_sqdist(const double* X, int d, const double* Q, int64_t npairs,
                     const int32_t* qrow, const int32_t* xcol, double* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npairs; ++k)
        out[k] = sqdist(Q + (size_t)qrow[k] * d, X + (size_t)xcol[k] * d, d);
}

/* ---------------------------------------------------------------------------
 * Nerve 1-skeleton (Sec. 2.1, Sec. 5.2): for landmark ordinals i < j the edge
 * exists iff the sorted membership lists of rows i and j share an id.
 *
 * With prune != 0, pairs whose landmarks are at squared distance above
 * 4*eps2 (with a relative margin of 1e-9) are skipped without intersecting:
 * a common member x would give d(l_i,l_j) <= d(l_i,x) + d(x,l_j) < 2 eps by
 * the triangle inequality (metric axiom 4, Sec. 2.1), so such pairs have no
 * edge.  The tests check that pruning changes nothing.
 *
 * Two phases: edges == NULL counts per row i into row_counts (length L);
 * otherwise edges (2 ints per edge, lexicographic) are written at
 * row_offsets[i].
 * ------------------------------------------------------------------------- */
static int lists_intersect(const int32_t* a, int64_t na, const int32_t* b, int64_t nb) {
    int64_t p = 0, q = 0;
    while (p < na && q < nb) {
        if (a[p] == b[q]) return 1;
        if (a[p] < b[q]) ++p; else ++q;
    }
    return 0;
}

void bmo_edges(const double* X, int d, const int32_t* landmarks, int64_t L, double eps2,
               const int64_t* offsets, const int32_t* ids, int prune,
               int64_t* row_counts, const int64_t* row_offsets, int32_t* edges) {
    const double lim = 4.0 * eps2 * (1.0 + 1e-9);
    #pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < L; ++i) {
        const double* li = X + (size_t)landmarks[i] * d;
        int64_t c = 0;
        int64_t o = edges ? row_offsets[i] : 0;
        for (int64_t j = i + 1; j < L; ++j) {
            if (prune && sqdist(li, X + (size_t)landmarks[j] * d, d) > lim) continue;
            if (lists_intersect(ids + offsets[i], offsets[i + 1] - offsets[i],
                                ids + offsets[j], offsets[j + 1] - offsets[j])) {
                if (edges) {
                    edges[2 * o] = (int32_t)i;
                    edges[2 * o + 1] = (int32_t)j;
                    ++o;
                } else {
                    ++c;
                }
            }
        }
        if (!edges) row_counts[i] = c;
    }
}

/* ---------------------------------------------------------------------------
 * Target-occupancy scale, Sec. 6.1: for each point the distance to its k-th
 * nearest neighbour, the point itself counted as the first.  Brute force:
 * all n squared distances of the row, then the k-th smallest by selection.
 * out[i] = sqrt(k-th smallest D(X_i, .)).
 * ------------------------------------------------------------------------- */
static double kth_smallest(double* v, int64_t n, int64_t k /* 0-based */) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        double pivot = v[lo + (hi - lo) / 2];
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (v[i] < pivot) ++i;
            while (v[j] > pivot) --j;
            if (i <= j) { double t = v[i]; v[i] = v[j]; v[j] = t; ++i; --j; }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return v[k];
    }
    return v[k];
}

int bmo_kth_nn_dist(const double* X, int64_t n, int d, int64_t k, double* out) {
    if (k < 1 || k > n) return -1;
    int bad = 0;
    #pragma omp parallel
    {
        double* row = (double*)malloc(sizeof(double) * (size_t)n);
        if (!row) {
            #pragma omp atomic write
            bad = 1;
        }
        #pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            if (!row) continue;
            const double* p = X + (size_t)i * d;
            for (int64_t j = 0; j < n; ++j) row[j] = sqdist(p, X + (size_t)j * d, d);
            out[i] = sqrt(kth_smallest(row, n, k - 1));
        }
        free(row);
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * Ball tree, Sec. 3.1.  Node centre c_i = (max_i + min_i)/2 over its points;
 * radius R = max_x d(c, x); split by p_A = farthest point from c and
 * p_B = farthest point from p_A; a point goes to X_A when it is closer to p_A
 * than to p_B, otherwise (ties included) to X_B.  Recursion stops when the
 * node holds at most leaf_size points, or the split leaves a side empty
 * (all points identical).
 *
 * Range query: a node is discarded when d(q,c) - R > r (triangle
 * inequality); a margin of 1e-9 (R + r) keeps FP64 square-root rounding from
 * discarding a true member.  Leaves are scanned with the exact test
 * D(q,x) < r^2, the same test as the brute-force oracle.
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t begin, end;     /* range in the permutation array */
    int32_t left, right;    /* child node ids, -1 for leaves  */
    double radius;
    int64_t centre;         /* offset of the centre in the centre pool */
} bt_node;

typedef struct {
    const double* X;
    int d;
    int64_t n;
    int32_t* perm;
    bt_node* nodes;
    int64_t n_nodes, cap_nodes;
    double* centres;
    int leaf_size;
} bt_tree;

static int64_t bt_new_node(bt_tree* t) {
    if (t->n_nodes == t->cap_nodes) {
        int64_t nc = t->cap_nodes ? 2 * t->cap_nodes : 64;
        bt_node* nn = (bt_node*)realloc(t->nodes, sizeof(bt_node) * (size_t)nc);
        double* cc = (double*)realloc(t->centres, sizeof(double) * (size_t)nc * (size_t)t->d);
        if (!nn || !cc) { if (nn) t->nodes = nn; if (cc) t->centres = cc; return -1; }
        t->nodes = nn; t->centres = cc; t->cap_nodes = nc;
    }
    return t->n_nodes++;
}

static int bt_build_node(bt_tree* t, int64_t begin, int64_t end) {
    int64_t id = bt_new_node(t);
    if (id < 0) return -1;
    const int d = t->d;
    const double* X = t->X;
    int32_t* perm = t->perm;
    double* c = t->centres + (size_t)id * d;
    for (int i = 0; i < d; ++i) {
        double mx = -INFINITY, mn = INFINITY;
        for (int64_t p = begin; p < end; ++p) {
            double v = X[(size_t)perm[p] * d + i];
            if (v > mx) mx = v;
            if (v < mn) mn = v;
        }
        c[i] = (mx + mn) / 2.0;
    }
    double r2 = 0.0;
    int64_t pa = begin;
    for (int64_t p = begin; p < end; ++p) {
        double s = sqdist(c, X + (size_t)perm[p] * d, d);
        if (s > r2) { r2 = s; pa = p; }
    }
    bt_node* nd = &t->nodes[id];
    nd->begin = begin; nd->end = end; nd->left = nd->right = -1;
    nd->radius = sqrt(r2);
    nd->centre = id * d;
    if (end - begin <= t->leaf_size || r2 == 0.0) return (int)id;

    const double* xa = X + (size_t)perm[pa] * d;
    double far2 = -1.0;
    int64_t pb = begin;
    for (int64_t p = begin; p < end; ++p) {
        double s = sqdist(xa, X + (size_t)perm[p] * d, d);
        if (s > far2) { far2 = s; pb = p; }
    }
    const double* xb = X + (size_t)perm[pb] * d;
    /* stable partition: X_A first (closer to p_A), then X_B */
    int64_t cnt = end - begin;
    int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)cnt);
    if (!tmp) return -1;
    int64_t na = 0, nb = 0;
    for (int64_t p = begin; p < end; ++p) {
        const double* xp = X + (size_t)perm[p] * d;
        if (sqdist(xp, xa, d) < sqdist(xp, xb, d)) perm[begin + na++] = perm[p];
        else tmp[nb++] = perm[p];
    }
    memcpy(perm + begin + na, tmp, sizeof(int32_t) * (size_t)nb);
    free(tmp);
    if (na == 0 || nb == 0) return (int)id;   /* cannot split further */
    int l = bt_build_node(t, begin, begin + na);
    if (l < 0) return -1;
    int r = bt_build_node(t, begin + na, end);
    if (r < 0) return -1;
    t->nodes[id].left = l;
    t->nodes[id].right = r;
    return (int)id;
}

void* bmo_bt_build(const double* X, int64_t n, int d, int leaf_size) {
    bt_tree* t = (bt_tree*)calloc(1, sizeof(bt_tree));
    if (!t) return NULL;
    t->X = X; t->d = d; t->n = n; t->leaf_size = leaf_size > 0 ? leaf_size : 40;
    t->perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!t->perm) { free(t); return NULL; }
    for (int64_t i = 0; i < n; ++i) t->perm[i] = (int32_t)i;
    if (n > 0 && bt_build_node(t, 0, n) < 0) {
        free(t->perm); free(t->nodes); free(t->centres); free(t);
        return NULL;
    }
    return t;
}

void bmo_bt_free(void* h) {
    bt_tree* t = (bt_tree*)h;
    if (!t) return;
    free(t->perm); free(t->nodes); free(t->centres); free(t);
}

int64_t bmo_bt_node_count(void* h) { return ((bt_tree*)h)->n_nodes; }

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Members of R_r(q) via the tree; returns the count, writes at most cap ids
 * (sorted ascending when all fit).  Iterative traversal with an explicit stack. */
static int64_t bt_query(const bt_tree* t, const double* q, double r, double r2,
                        int32_t* out, int64_t cap) {
    if (t->n == 0) return 0;
    /* a depth-first stack never holds more entries than there are nodes */
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)(t->n_nodes + 1));
    if (!stack) return -1;
    int64_t sp = 0;
    int64_t cnt = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const bt_node* nd = &t->nodes[stack[--sp]];
        double dc = sqrt(sqdist(q, t->centres + nd->centre, t->d));
        if (dc - nd->radius > r + 1e-9 * (nd->radius + r)) continue;   /* pruned */
        if (nd->left < 0) {
            for (int64_t p = nd->begin; p < nd->end; ++p) {
                int32_t id = t->perm[p];
                if (sqdist(q, t->X + (size_t)id * t->d, t->d) < r2) {
                    if (cnt < cap) out[cnt] = id;
                    ++cnt;
                }
            }
        } else {
            stack[sp++] = nd->right;
            stack[sp++] = nd->left;
        }
    }
    free(stack);
    if (cnt <= cap) qsort(out, (size_t)cnt, sizeof(int32_t), cmp_i32);
    return cnt;
}

/* Batched ball-tree range queries, two phases like bmo_range_count/fill. */
int bmo_bt_range_count(void* h, const double* Q, int64_t m, double r, int64_t* counts) {
    const bt_tree* t = (const bt_tree*)h;
    int bad = 0;
    const double r2 = r * r;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < m; ++j) {
        int64_t c = bt_query(t, Q + (size_t)j * t->d, r, r2, NULL, 0);
        if (c < 0) {
            #pragma omp atomic write
            bad = 1;
        }
        counts[j] = c;
    }
    return bad ? -1 : 0;
}

int bmo_bt_range_fill(void* h, const double* Q, int64_t m, double r, const int64_t* offsets,
                      int32_t* ids) {
    const bt_tree* t = (const bt_tree*)h;
    int bad = 0;
    const double r2 = r * r;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < m; ++j) {
        int64_t cap = offsets[j + 1] - offsets[j];
        int64_t c = bt_query(t, Q + (size_t)j * t->d, r, r2, ids + offsets[j], cap);
        if (c != cap) {
            #pragma omp atomic write
            bad = 1;
        }
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * Verified range set over a candidate set (Sec. 5.3): the candidates of query j
 * are the points whose cell is one of the query's probed cells; a candidate is
 * returned iff D(Q_j, X_i) < eps2.  cell_of[i] in [0, nlist), probes: m x nprobe.
 * Two phases like bmo_range_count / bmo_range_fill.
 * ------------------------------------------------------------------------- */
static void mark_probes(unsigned char* flag, int nlist, const int32_t* probes, int nprobe, int64_t j) {
    memset(flag, 0, (size_t)nlist);
    for (int k = 0; k < nprobe; ++k) {
        int32_t c = probes[(size_t)j * nprobe + k];
        if (c >= 0 && c < nlist) flag[c] = 1;
    }
}

int bmo_masked_range_count(const double* X, int64_t n, int d, const double* Q, int64_t m, double eps2,
                           const int32_t* cell_of, int nlist, const int32_t* probes, int nprobe, int64_t* counts) {
    int bad = 0;
    #pragma omp parallel
    {
        unsigned char* flag = (unsigned char*)malloc((size_t)nlist);
        if (!flag) {
            #pragma omp atomic write
            bad = 1;
        }
        #pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < m; ++j) {
            if (!flag) continue;
            mark_probes(flag, nlist, probes, nprobe, j);
            const double* q = Q + (size_t)j * d;
            int64_t c = 0;
            for (int64_t i = 0; i < n; ++i)
                if (flag[cell_of[i]] && sqdist(q, X + (size_t)i * d, d) < eps2) ++c;
            counts[j] = c;
        }
        free(flag);
    }
    return bad ? -1 : 0;
}

int bmo_masked_range_fill(const double* X, int64_t n, int d, const double* Q, int64_t m, double eps2,
                          const int32_t* cell_of, int nlist, const int32_t* probes, int nprobe,
                          const int64_t* offsets, int32_t* ids) {
    int bad = 0;
    #pragma omp parallel
    {
        unsigned char* flag = (unsigned char*)malloc((size_t)nlist);
        if (!flag) {
            #pragma omp atomic write
            bad = 1;
        }
        #pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < m; ++j) {
            if (!flag) continue;
            mark_probes(flag, nlist, probes, nprobe, j);
            const double* q = Q + (size_t)j * d;
            int64_t o = offsets[j];
            for (int64_t i = 0; i < n; ++i)
                if (flag[cell_of[i]] && sqdist(q, X + (size_t)i * d, d) < eps2) ids[o++] = (int32_t)i;
        }
        free(flag);
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * Farthest point sampling, Sec. 2.2.  L = {first}; repeat: for every point x
 * the distance to the set, m(x) = min_{l in L} D(x,l) (kept up to date with
 * each new landmark); x* = argmax_x m(x), the smallest index among equal
 * maxima; x* joins L when m(x*) >= eps^2, otherwise the procedure stops.
 * Reading: the paper writes "> eps"; with open balls (a point at distance
 * exactly eps is not covered) ">=" is the rule under which every point ends
 * inside an open ball, the same cover condition as the greedy.
 * Returns the number of landmarks (written in selection order), -1 on an
 * allocation failure.
 * ------------------------------------------------------------------------- */
int64_t bmo_fps(const double* X, int64_t n, int d, double eps2, int64_t first, int32_t* landmarks) {
    if (n <= 0) return 0;
    double* m = (double*)malloc(sizeof(double) * (size_t)n);
    if (!m) return -1;
    for (int64_t x = 0; x < n; ++x) m[x] = INFINITY;
    int64_t L = 0;
    int64_t cur = first;
    landmarks[L++] = (int32_t)cur;
    while (1) {
        const double* c = X + (size_t)cur * d;
        #pragma omp parallel for schedule(static)
        for (int64_t x = 0; x < n; ++x) {
            const double D = sqdist(X + (size_t)x * d, c, d);
            if (D < m[x]) m[x] = D;
        }
        int64_t best = 0;
        for (int64_t x = 1; x < n; ++x)
            if (m[x] > m[best]) best = x;
        if (!(m[best] >= eps2)) break;
        if (L >= n) break;   /* never reached for eps > 0: a landmark is at distance 0 */
        cur = best;
        landmarks[L++] = (int32_t)cur;
    }
    free(m);
    return L;
}

/* ---------------------------------------------------------------------------
 * Coloring, Sec. 2.3: c(l_i) = statistic of f over X_i, the ids of CSR row i.
 *   stat 0: mean, (sum of f over the row, in row order, FP64) / |X_i|
 *   stat 1: median (numpy's rule: the middle value, or for an even count the
 *           mean of the two middle values computed as (a + b) / 2)
 *   stat 2: minimum, stat 3: maximum
 * An empty row gets NaN.  Returns -1 on an allocation failure.
 * ------------------------------------------------------------------------- */
static int cmp_f64(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

int bmo_color(const int64_t* offsets, const int32_t* ids, int64_t rows, const double* f, int stat, double* out) {
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < rows; ++r) {
        const int64_t b = offsets[r], e = offsets[r + 1], cnt = e - b;
        if (cnt == 0) {
            out[r] = NAN;
            continue;
        }
        if (stat == 0) {
            double sum = 0.0;
            for (int64_t j = b; j < e; ++j) sum += f[ids[j]];
            out[r] = sum / (double)cnt;
        } else if (stat == 1) {
            double* v = (double*)malloc(sizeof(double) * (size_t)cnt);
            if (!v) {
                #pragma omp atomic write
                bad = 1;
                continue;
            }
            for (int64_t j = b; j < e; ++j) v[j - b] = f[ids[j]];
            qsort(v, (size_t)cnt, sizeof(double), cmp_f64);
            out[r] = (cnt % 2) ? v[cnt / 2] : (v[cnt / 2 - 1] + v[cnt / 2]) / 2.0;
            free(v);
        } else {
            double best = f[ids[b]];
            for (int64_t j = b + 1; j < e; ++j) {
                const double x = f[ids[j]];
                if (stat == 2 ? x < best : x > best) best = x;
            }
            out[r] = best;
        }
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * Proximity graph and graph range query (Sec. 5.4: the candidate set C(q) of a
 * non-exhaustive index is what a partial graph traversal visits; membership is
 * then decided with the exact distance, so no false positives).
 *
 * Graph: for every point i its M nearest other points by (D, id), D the FP64
 * squared distance; the undirected union of those arcs; each adjacency list
 * ascending by id (CSR adj_off / adj).
 *
 * Query q (all distances FP64 D, candidates ordered by (D, id)):
 *   1. entry: the nearest of the E entry points e_t = floor(t n / E), t < E;
 *   2. beam: a list R of at most ef visited nodes, the best by (D, id), each
 *      flagged expanded or not; repeatedly expand the best unexpanded node of R
 *      (visit its neighbours in adjacency order: a neighbour not yet visited is
 *      visited, and enters R when R has room or it beats R's worst, which then
 *      leaves R); stop when every node of R is expanded;
 *   3. range expansion: every visited node with D < eps^2 that was not expanded
 *      is expanded in order of visit (first in, first out), visiting its
 *      neighbours; those with D < eps^2 join the queue;
 *   at most max_visits nodes are visited per query (visits stop at the cap).
 * Row j = { visited v : D(q_j, v) < eps^2 }, ascending.
 * ------------------------------------------------------------------------- */
typedef struct { double D; int32_t id; } dkey;

static int dkey_less(dkey a, dkey b) { return a.D < b.D || (a.D == b.D && a.id < b.id); }

int bmo_knn_graph(const double* X, int64_t n, int d, int M, int32_t* nbr) {
    if (M < 1 || M >= n) return -1;
    int bad = 0;
    #pragma omp parallel
    {
        dkey* best = (dkey*)malloc(sizeof(dkey) * (size_t)(M + 1));
        if (!best) {
            #pragma omp atomic write
            bad = 1;
        }
        #pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            if (!best) continue;
            int cnt = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                dkey c = {sqdist(X + (size_t)i * d, X + (size_t)j * d, d), (int32_t)j};
                if (cnt == M && !dkey_less(c, best[M - 1])) continue;
                int p = cnt < M ? cnt++ : M - 1;           /* insertion into the sorted best list */
                while (p > 0 && dkey_less(c, best[p - 1])) { best[p] = best[p - 1]; --p; }
                best[p] = c;
            }
            for (int t = 0; t < M; ++t) nbr[(size_t)i * M + t] = best[t].id;
        }
        free(best);
    }
    return bad ? -1 : 0;
}

typedef struct {
    int32_t* mark;       /* n: visit stamp (query index + 1) */
    int32_t* visited;    /* visit order */
    double* vd;          /* D of the visited nodes */
    unsigned char* expd; /* expanded flag per visited slot */
    int32_t* slot;       /* n: visited slot of a node (valid when marked) */
    dkey* R;             /* beam, sorted */
    int32_t* Rslot;
} gq_work;

/* one query; writes the in-range ids (ascending) to out (when non-NULL), returns their count */
static int64_t graph_query(const double* X, int64_t n, int d, const int64_t* adj_off, const int32_t* adj,
                           const double* q, double eps2, int E, int ef, int64_t max_visits, int32_t stamp,
                           gq_work* w, int32_t* out) {
    int64_t nv = 0;
    /* 1. entry */
    int64_t start = 0;
    double bd = INFINITY;
    for (int t = 0; t < E; ++t) {
        const int64_t e = (int64_t)t * n / E;
        const double D = sqdist(q, X + (size_t)e * d, d);
        if (D < bd || (D == bd && e < start)) { bd = D; start = e; }
    }
    w->mark[start] = stamp;
    w->slot[start] = (int32_t)nv;
    w->visited[nv] = (int32_t)start;
    w->vd[nv] = bd;
    w->expd[nv] = 0;
    ++nv;
    int nR = 1;
    w->R[0].D = bd;
    w->R[0].id = (int32_t)start;
    w->Rslot[0] = 0;
    /* 2. beam */
    while (1) {
        int pick = -1;
        for (int r = 0; r < nR; ++r)
            if (!w->expd[w->Rslot[r]]) { pick = r; break; }
        if (pick < 0) break;
        const int32_t c = w->R[pick].id;
        w->expd[w->Rslot[pick]] = 1;
        for (int64_t a = adj_off[c]; a < adj_off[c + 1] && nv < max_visits; ++a) {
            const int32_t v = adj[a];
            if (w->mark[v] == stamp) continue;
            const double D = sqdist(q, X + (size_t)v * d, d);
            w->mark[v] = stamp;
            w->slot[v] = (int32_t)nv;
            w->visited[nv] = v;
            w->vd[nv] = D;
            w->expd[nv] = 0;
            dkey k = {D, v};
            if (nR < ef || dkey_less(k, w->R[nR - 1])) {
                int p = nR < ef ? nR++ : nR - 1;
                while (p > 0 && dkey_less(k, w->R[p - 1])) { w->R[p] = w->R[p - 1]; w->Rslot[p] = w->Rslot[p - 1]; --p; }
                w->R[p] = k;
                w->Rslot[p] = (int32_t)nv;
            }
            ++nv;
        }
    }
    /* 3. range expansion, first in first out over the visit order */
    for (int64_t h = 0; h < nv; ++h) {
        if (!(w->vd[h] < eps2) || w->expd[h]) continue;
        w->expd[h] = 1;
        const int32_t c = w->visited[h];
        for (int64_t a = adj_off[c]; a < adj_off[c + 1] && nv < max_visits; ++a) {
            const int32_t v = adj[a];
            if (w->mark[v] == stamp) continue;
            w->mark[v] = stamp;
            w->slot[v] = (int32_t)nv;
            w->visited[nv] = v;
            w->vd[nv] = sqdist(q, X + (size_t)v * d, d);
            w->expd[nv] = 0;
            ++nv;
        }
    }
    int64_t cnt = 0;
    for (int64_t h = 0; h < nv; ++h)
        if (w->vd[h] < eps2) {
            if (out) out[cnt] = w->visited[h];
            ++cnt;
        }
    if (out) qsort(out, (size_t)cnt, sizeof(int32_t), cmp_i32);
    return cnt;
}

/* counts (pass offsets == NULL) or fills (ids at offsets[j]) the rows of every query */
int bmo_graph_range(const double* X, int64_t n, int d, const int64_t* adj_off, const int32_t* adj,
                    const double* Q, int64_t m, double eps2, int E, int ef, int64_t max_visits,
                    int64_t* counts, const int64_t* offsets, int32_t* ids) {
    if (n <= 0 || E < 1 || ef < 1 || max_visits < 1) return -1;
    if (E > n) E = (int)n;
    int bad = 0;
    #pragma omp parallel
    {
        gq_work w;
        w.mark = (int32_t*)calloc((size_t)n, sizeof(int32_t));
        w.slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        w.visited = (int32_t*)malloc(sizeof(int32_t) * (size_t)(max_visits + 1));
        w.vd = (double*)malloc(sizeof(double) * (size_t)(max_visits + 1));
        w.expd = (unsigned char*)malloc((size_t)(max_visits + 1));
        w.R = (dkey*)malloc(sizeof(dkey) * (size_t)ef);
        w.Rslot = (int32_t*)malloc(sizeof(int32_t) * (size_t)ef);
        const int ok = w.mark && w.slot && w.visited && w.vd && w.expd && w.R && w.Rslot;
        if (!ok) {
            #pragma omp atomic write
            bad = 1;
        }
        #pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < m; ++j) {
            if (!ok) continue;
            const int64_t c = graph_query(X, n, d, adj_off, adj, Q + (size_t)j * d, eps2, E, ef, max_visits,
                                          (int32_t)(j + 1), &w, offsets ? ids + offsets[j] : NULL);
            if (counts) counts[j] = c;
        }
        free(w.mark); free(w.slot); free(w.visited); free(w.vd); free(w.expd); free(w.R); free(w.Rslot);
    }
    return bad ? -1 : 0;
}
