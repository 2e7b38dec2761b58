/*
 * Oracle for Localized Topological Simplification (LTS) on Freudenthal grids.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded CPU
 * restatement of the method, written to be checked against the paper by eye.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * What follows the paper, and where:
 *   - domain, star/link, lower/upper link, critical point index ....... Sec. 3.1
 *   - persistence pairs by the Elder rule (input selector) ............ Sec. 3.3
 *   - order field (sort by value, ties by memory position) ............ Sec. 4.1
 *     (float32 fields, and float64 fields through orc_lts_f64)
 *   - superlevel set propagation from one maximum (step 1) ............ Sec. 4.2
 *   - hill chains: stop / merge at saddles, queue melding, union-find . Sec. 4.3
 *   - arrival counter of unvisited higher neighbours .................. Sec. 4.4
 *   - localized simplification by alternating propagations (step 2) .. Sec. 4.2, Eq. 3-5
 *   - local to global order (step 3), pair order ...................... Sec. 4.2, Eq. 6
 *   - symbolic to numerical perturbation (step 4) ..................... Sec. 4.2
 *   - minima processed symmetrically to maxima ........................ Sec. 4
 *   - persistence-driven selection by eps-bounded propagations ........ Sec. 4.5
 *
 * Readings taken where the paper is silent (each is listed in the design
 * notes of the repository):
 *   - the triangulation is Freudenthal/Kuhn with diagonals along +(1,1)
 *     and +(1,1,1); a missing neighbour at the grid boundary is dropped;
 *   - -0.0 and +0.0 are one value (ties by vertex id); NaN is an error;
 *   - "higher neighbour visited by some propagation" (Sec. 4.3) is read as
 *     "owned by a propagation that has arrived at this saddle": the counter
 *     of Sec. 4.4 counts the higher neighbours whose class has not yet
 *     arrived.  The same regions are given by a join-tree sweep (method B);
 *   - the vertex set to minus infinity in step 2 is, among the vertices of
 *     R other than s that have a neighbour outside R and whose removal
 *     leaves R connected, the one with the lowest order (with a cut vertex
 *     the first propagation would not end there and could leave no
 *     authorized minimum);
 *   - the sublevel propagation of step 2 starts, as the paper says, from
 *     the current authorized minima (minima of the current local order with
 *     a neighbour outside R).  Taken literally the alternation can cycle
 *     for ever (a cluster hanging off a cut vertex swaps its stray minimum
 *     and maximum at every iteration); a region whose literal alternation
 *     has not ended after 2|R|+2 propagations (or that has no authorized
 *     minimum to start from) is redone from the first propagation's order
 *     with every vertex allowed to be a minimum (all of R other than s with
 *     an outside neighbour) as seeds, which always ended;
 *   - the pair order of Eq. 6 is made total for regions sharing a saddle:
 *     sibling blocks are ordered by the order of their highest vertex;
 *   - the numerical perturbation uses zeta = 0: every region vertex takes the
 *     saddle's value bit for bit;
 *   - one minima pass, then one maxima pass;
 *   - the optional restoration of swallowed authorized extrema (Sec. 4.2
 *     step 3, mode flag ORC_MODE_RESTORE): each one moves below the other
 *     vertices of its region's block, in increasing order, unless that would
 *     leave one of its neighbours without a higher neighbour (a new maximum);
 *   - persistence-driven selection (Sec. 4.5): eps is absolute; the tracked
 *     difference is f(m) - f(v) (minima pass: f(v) - f(m)) for the class's
 *     highest extremum m and the vertex v about to be taken, in double
 *     precision from the float32 values; the propagation ends when it is
 *     strictly greater than eps, before v is taken; a class whose queue runs
 *     dry holds the global extremum, which is kept; each pass selects on the
 *     field it receives.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NAN 2
#define ORC_ERR_NO_AUTHORIZED 3
#define ORC_ERR_OOM 4
#define ORC_ERR_INTERNAL 7

#define ORC_MODE_MIN 1
#define ORC_MODE_MAX 2
#define ORC_MODE_BOTH 3
#define ORC_MODE_RESTORE 4   /* or-ed into the mode: restore swallowed authorized extrema */

typedef struct {
    int64_t n_vertices;
    int64_t removed[2];          /* [0] minima pass, [1] maxima pass: unauthorized extrema */
    int64_t regions[2];          /* regions (one per hill chain)                          */
    int64_t region_vertices[2];  /* vertices moved (region members, saddles excluded)     */
    int64_t max_region[2];       /* largest region, members only                          */
    int32_t max_local_floods[2]; /* most propagations any region needed in step 2         */
    int32_t pad;
    int64_t total_local_floods[2];
    int64_t fallback_regions[2]; /* regions step 2 redid with all-boundary seeds            */
    int64_t restored[2];         /* swallowed authorized extrema restored (mode RESTORE)     */
} orc_stats;

/* ------------------------------------------------------------------------ */
/* Domain: regular grid with the Freudenthal (Kuhn) triangulation.          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int ndim;
    int64_t X, Y, Z, n;
    int nn;
    int off[14][3];
} grid_t;

/* The neighbours of a vertex are the lattice points p with p-v in {0,1}^d or
 * in -{0,1}^d (v excluded): every such segment is an edge of the Kuhn
 * triangulation of the unit cubes. */
static void make_offsets(grid_t* G) {
    int k = 0;
    int d = G->ndim;
    for (int m = 1; m < (1 << d); ++m) {
        int o[3] = {0, 0, 0};
        for (int b = 0; b < d; ++b) o[b] = (m >> b) & 1;
        G->off[k][0] = o[0]; G->off[k][1] = o[1]; G->off[k][2] = o[2];
        ++k;
    }
    int half = k;
    for (int i = 0; i < half; ++i) {
        G->off[k][0] = -G->off[i][0]; G->off[k][1] = -G->off[i][1]; G->off[k][2] = -G->off[i][2];
        ++k;
    }
    G->nn = k;
}

static int grid_init(grid_t* G, int ndim, const int64_t* dims) {
    if (ndim != 2 && ndim != 3) return ORC_ERR_ARG;
    G->ndim = ndim;
    G->X = dims[0]; G->Y = dims[1]; G->Z = (ndim == 3) ? dims[2] : 1;
    if (G->X < 2 || G->Y < 2 || (ndim == 3 && G->Z < 2)) return ORC_ERR_ARG;
    G->n = G->X * G->Y * G->Z;
    if (G->n >= ((int64_t)1 << 31)) return ORC_ERR_ARG;
    make_offsets(G);
    return ORC_OK;
}

/* Existing neighbours of v, in offset order; returns their count. */
static int nbrs(const grid_t* G, int64_t v, int32_t* out) {
    int64_t x = v % G->X, y = (v / G->X) % G->Y, z = v / (G->X * G->Y);
    int c = 0;
    for (int k = 0; k < G->nn; ++k) {
        int64_t a = x + G->off[k][0], b = y + G->off[k][1], e = z + G->off[k][2];
        if (a < 0 || a >= G->X || b < 0 || b >= G->Y || e < 0 || e >= G->Z) continue;
        out[c++] = (int32_t)(a + G->X * (b + G->Y * e));
    }
    return c;
}

/* Same, but also reports which offset each neighbour came from. */
static int nbrs_k(const grid_t* G, int64_t v, int32_t* out, int* kk) {
    int64_t x = v % G->X, y = (v / G->X) % G->Y, z = v / (G->X * G->Y);
    int c = 0;
    for (int k = 0; k < G->nn; ++k) {
        int64_t a = x + G->off[k][0], b = y + G->off[k][1], e = z + G->off[k][2];
        if (a < 0 || a >= G->X || b < 0 || b >= G->Y || e < 0 || e >= G->Z) continue;
        kk[c] = k;
        out[c++] = (int32_t)(a + G->X * (b + G->Y * e));
    }
    return c;
}

/* A set of lattice points is a simplex of the Kuhn triangulation iff the
 * points form a chain under the componentwise order and the last minus the
 * first lies in {0,1}^d. */
static int is_kuhn_simplex(int d, int cnt, const int (*pts)[3]) {
    int idx[4] = {0, 1, 2, 3};
    /* sort by coordinate sum (insertion sort, at most four points) */
    for (int i = 1; i < cnt; ++i) {
        int j = i;
        while (j > 0) {
            const int* p = pts[idx[j - 1]];
            const int* q = pts[idx[j]];
            if (p[0] + p[1] + p[2] > q[0] + q[1] + q[2]) {
                int t = idx[j]; idx[j] = idx[j - 1]; idx[j - 1] = t; --j;
            } else break;
        }
    }
    for (int i = 1; i < cnt; ++i) {
        const int* p = pts[idx[i - 1]];
        const int* q = pts[idx[i]];
        int same = 1;
        for (int b = 0; b < d; ++b) {
            if (q[b] < p[b]) return 0;
            if (q[b] != p[b]) same = 0;
        }
        if (same) return 0;
    }
    const int* lo = pts[idx[0]];
    const int* hi = pts[idx[cnt - 1]];
    for (int b = 0; b < d; ++b) {
        int df = hi[b] - lo[b];
        if (df != 0 && df != 1) return 0;
    }
    return 1;
}

/* Link graph of an interior vertex: pairs of offsets (a,b) with {0,a,b} a
 * simplex.  Writes pairs of offset indices; returns the number of edges. */
int orc_link_edges(int ndim, int32_t* pairs) {
    grid_t G; memset(&G, 0, sizeof G); G.ndim = ndim; make_offsets(&G);
    int e = 0;
    for (int i = 0; i < G.nn; ++i)
        for (int j = i + 1; j < G.nn; ++j) {
            int pts[3][3] = {{0, 0, 0},
                             {G.off[i][0], G.off[i][1], G.off[i][2]},
                             {G.off[j][0], G.off[j][1], G.off[j][2]}};
            if (is_kuhn_simplex(ndim, 3, (const int (*)[3])pts)) {
                if (pairs) { pairs[2 * e] = i; pairs[2 * e + 1] = j; }
                ++e;
            }
        }
    return e;
}

/* Triangles of the link (3D): triples of offsets (a,b,c) with {0,a,b,c} a
 * tetrahedron of the triangulation. */
int orc_link_triangles(int ndim, int32_t* tris) {
    grid_t G; memset(&G, 0, sizeof G); G.ndim = ndim; make_offsets(&G);
    int t = 0;
    for (int i = 0; i < G.nn; ++i)
        for (int j = i + 1; j < G.nn; ++j)
            for (int k = j + 1; k < G.nn; ++k) {
                int pts[4][3] = {{0, 0, 0},
                                 {G.off[i][0], G.off[i][1], G.off[i][2]},
                                 {G.off[j][0], G.off[j][1], G.off[j][2]},
                                 {G.off[k][0], G.off[k][1], G.off[k][2]}};
                if (is_kuhn_simplex(ndim, 4, (const int (*)[3])pts)) {
                    if (tris) { tris[3 * t] = i; tris[3 * t + 1] = j; tris[3 * t + 2] = k; }
                    ++t;
                }
            }
    return t;
}

int orc_neighbour_offsets(int ndim, int32_t* off) {
    grid_t G; memset(&G, 0, sizeof G); G.ndim = ndim; make_offsets(&G);
    for (int k = 0; k < G.nn; ++k)
        for (int b = 0; b < 3; ++b) off[3 * k + b] = G.off[k][b];
    return G.nn;
}

/* ------------------------------------------------------------------------ */
/* Order field (Sec. 4.1): vertices sorted by increasing f, equal values     */
/* disambiguated by their position in memory; O(v) is the rank of v.        */
/* ------------------------------------------------------------------------ */

static const float* s_sort_f;
static int cmp_value_then_id(const void* pa, const void* pb) {
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    float fa = s_sort_f[a], fb = s_sort_f[b];
    if (fa < fb) return -1;        /* IEEE compare: -0.0 == +0.0 */
    if (fa > fb) return 1;
    return (a > b) - (a < b);
}

int orc_order_field(int ndim, const int64_t* dims, const float* f, int32_t* O) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    for (int64_t v = 0; v < G.n; ++v)
        if (isnan(f[v])) return ORC_ERR_NAN;
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * G.n);
    if (!idx) return ORC_ERR_OOM;
    for (int64_t v = 0; v < G.n; ++v) idx[v] = (int32_t)v;
    s_sort_f = f;
    qsort(idx, (size_t)G.n, sizeof(int32_t), cmp_value_then_id);
    for (int64_t i = 0; i < G.n; ++i) O[idx[i]] = (int32_t)i;
    free(idx);
    return ORC_OK;
}

/* The same for a float64 field. */
static const double* s_sort_d;
static int cmp_dvalue_then_id(const void* pa, const void* pb) {
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    double fa = s_sort_d[a], fb = s_sort_d[b];
    if (fa < fb) return -1;        /* IEEE compare: -0.0 == +0.0 */
    if (fa > fb) return 1;
    return (a > b) - (a < b);
}

int orc_order_field_f64(int ndim, const int64_t* dims, const double* f, int32_t* O) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    for (int64_t v = 0; v < G.n; ++v)
        if (isnan(f[v])) return ORC_ERR_NAN;
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * G.n);
    if (!idx) return ORC_ERR_OOM;
    for (int64_t v = 0; v < G.n; ++v) idx[v] = (int32_t)v;
    s_sort_d = f;
    qsort(idx, (size_t)G.n, sizeof(int32_t), cmp_dvalue_then_id);
    for (int64_t i = 0; i < G.n; ++i) O[idx[i]] = (int32_t)i;
    free(idx);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Critical points (Sec. 3.1): numbers of connected components of the lower  */
/* and upper links.  Minimum: empty lower link; maximum: empty upper link;    */
/* regular: both non-empty and connected; otherwise a saddle.                */
/* ------------------------------------------------------------------------ */

static int small_find(int* p, int a) { while (p[a] != a) a = p[a]; return a; }

int orc_classify(int ndim, const int64_t* dims, const int32_t* O, int8_t* n_lower, int8_t* n_upper) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    int32_t pairs[2 * 64];
    int ne = orc_link_edges(ndim, pairs);
    for (int64_t v = 0; v < G.n; ++v) {
        int32_t nb[14]; int kk[14];
        int c = nbrs_k(&G, v, nb, kk);
        int present[14], lower[14], pos[14];
        for (int k = 0; k < 14; ++k) { present[k] = 0; lower[k] = 0; pos[k] = -1; }
        for (int i = 0; i < c; ++i) {
            present[kk[i]] = 1;
            lower[kk[i]] = O[nb[i]] < O[v];
            pos[kk[i]] = i;
        }
        for (int side = 0; side < 2; ++side) {
            int p[14];
            for (int k = 0; k < 14; ++k) p[k] = k;
            for (int e = 0; e < ne; ++e) {
                int a = pairs[2 * e], b = pairs[2 * e + 1];
                if (!present[a] || !present[b]) continue;
                int wa = side == 0 ? lower[a] : !lower[a];
                int wb = side == 0 ? lower[b] : !lower[b];
                if (wa && wb) {
                    int ra = small_find(p, a), rb = small_find(p, b);
                    if (ra != rb) p[ra] = rb;
                }
            }
            int comps = 0;
            for (int k = 0; k < G.nn; ++k) {
                if (!present[k]) continue;
                int w = side == 0 ? lower[k] : !lower[k];
                if (w && small_find(p, k) == k) ++comps;
            }
            if (side == 0) n_lower[v] = (int8_t)comps; else n_upper[v] = (int8_t)comps;
        }
        (void)pos;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Topological persistence (Sec. 3.3), used to select authorized extrema.   */
/* Maxima: components of the superlevel sets are born at maxima and merge at */
/* saddles; at a merge the component whose maximum is lower (the youngest)   */
/* dies, giving the pair <s, m> with persistence f(m) - f(s).  The global    */
/* maximum gets the function range.  Minima: the same on sublevel sets.      */
/* pers[v] is NaN for vertices that are not extrema of that kind.           */
/* ------------------------------------------------------------------------ */

static int64_t uf_find64(int64_t* p, int64_t a) {
    while (p[a] != a) { p[a] = p[p[a]]; a = p[a]; }
    return a;
}

static int persistence_one(const grid_t* G, const float* f, const int32_t* O,
                           const int32_t* perm, int descending, double* pers) {
    int64_t n = G->n;
    int64_t* par = (int64_t*)malloc(sizeof(int64_t) * n);
    int32_t* best = (int32_t*)malloc(sizeof(int32_t) * n);  /* extremum of component (at root) */
    if (!par || !best) { free(par); free(best); return ORC_ERR_OOM; }
    for (int64_t v = 0; v < n; ++v) { par[v] = -1; pers[v] = NAN; }
    double fmin = INFINITY, fmax = -INFINITY;
    for (int64_t v = 0; v < n; ++v) {
        if (f[v] < fmin) fmin = f[v];
        if (f[v] > fmax) fmax = f[v];
    }
    double range = fmax - fmin;
    for (int64_t i = 0; i < n; ++i) {
        int32_t v = descending ? perm[n - 1 - i] : perm[i];
        int32_t nb[14];
        int c = nbrs(G, v, nb);
        int64_t roots[14]; int nr = 0;
        for (int j = 0; j < c; ++j) {
            int32_t u = nb[j];
            int earlier = descending ? (O[u] > O[v]) : (O[u] < O[v]);
            if (!earlier) continue;
            int64_t r = uf_find64(par, u);
            int dup = 0;
            for (int q = 0; q < nr; ++q) if (roots[q] == r) dup = 1;
            if (!dup) roots[nr++] = r;
        }
        par[v] = v;
        if (nr == 0) { best[v] = v; continue; }       /* v is an extremum: birth */
        /* the oldest component survives (highest maximum / lowest minimum) */
        int64_t keep = roots[0];
        for (int q = 1; q < nr; ++q) {
            int32_t a = best[roots[q]], b = best[keep];
            int older = descending ? (O[a] > O[b]) : (O[a] < O[b]);
            if (older) keep = roots[q];
        }
        for (int q = 0; q < nr; ++q) {
            if (roots[q] == keep) continue;
            int32_t m = best[roots[q]];
            pers[m] = fabs((double)f[m] - (double)f[v]);
            par[roots[q]] = keep;
        }
        par[v] = keep;
    }
    /* the global extremum of this kind gets the function range */
    int32_t g = descending ? perm[n - 1] : perm[0];
    pers[g] = range;
    free(par); free(best);
    return ORC_OK;
}

int orc_persistence(int ndim, const int64_t* dims, const float* f, const int32_t* O,
                    double* pers_min, double* pers_max) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * G.n);
    if (!perm) return ORC_ERR_OOM;
    for (int64_t v = 0; v < G.n; ++v) perm[O[v]] = (int32_t)v;
    st = persistence_one(&G, f, O, perm, 0, pers_min);
    if (!st) st = persistence_one(&G, f, O, perm, 1, pers_max);
    free(perm);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Binary heap of (key, vertex), largest key first.                          */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t key; int32_t v; } hitem;
typedef struct { hitem* a; int64_t n, cap; } heap_t;

static int heap_push(heap_t* h, int64_t key, int32_t v) {
    if (h->n == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 16;
        hitem* na = (hitem*)realloc(h->a, sizeof(hitem) * nc);
        if (!na) return ORC_ERR_OOM;
        h->a = na; h->cap = nc;
    }
    int64_t i = h->n++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p].key >= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].key = key; h->a[i].v = v;
    return ORC_OK;
}

static hitem heap_pop(heap_t* h) {
    hitem top = h->a[0];
    hitem last = h->a[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        int64_t mk = last.key;
        if (l < h->n && h->a[l].key > mk) { m = l; mk = h->a[l].key; }
        if (r < h->n && h->a[r].key > mk) { m = r; }
        if (m == i) break;
        h->a[i] = h->a[m];
        i = m;
    }
    if (h->n > 0) h->a[i] = last;
    return top;
}

static void heap_free(heap_t* h) { free(h->a); h->a = NULL; h->n = h->cap = 0; }

/* meld: every entry of src goes into dst; src is emptied */
static int heap_meld(heap_t* dst, heap_t* src) {
    for (int64_t i = 0; i < src->n; ++i) {
        int st = heap_push(dst, src->a[i].key, src->a[i].v);
        if (st) return st;
    }
    heap_free(src);
    return ORC_OK;
}

/* small deterministic generator for the shuffled schedules (splitmix64) */
static uint64_t sm64(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------ */
/* Step 1 with hill chains, method A: one superlevel set propagation per     */
/* unauthorized maximum (Sec. 4.2 step 1, Sec. 4.3, Sec. 4.4).                */
/*                                                                            */
/* Everything works on an order field Od whose maxima are the extrema to     */
/* treat: Od = O for the maxima pass, Od = N-1-O for the minima pass.         */
/*                                                                            */
/* Output (canonical): regions sorted by (Od(saddle), Od(top)); region_of[v]  */
/* is the region of every member vertex (saddles excluded), -1 otherwise.     */
/* ------------------------------------------------------------------------ */

typedef struct {
    const grid_t* G;
    const int32_t* Od;
    int32_t* owner;     /* class that first popped the vertex, or -1 */
    int32_t* cnt;       /* higher neighbours whose class has not arrived; -1 = unset */
    int32_t* wait_head; /* classes waiting at the vertex (linked list), -1 = none */
    int32_t* wait_next;
    int32_t* parent;    /* union-find over classes */
    heap_t* heap;
} flood_t;

static int32_t cls_find(int32_t* p, int32_t a) {
    while (p[a] != a) { p[a] = p[p[a]]; a = p[a]; }
    return a;
}

static int push_lower_not_in(flood_t* F, int32_t v, int32_t c) {
    int32_t nb[14];
    int k = nbrs(F->G, v, nb);
    for (int j = 0; j < k; ++j) {
        int32_t u = nb[j];
        if (F->Od[u] >= F->Od[v]) continue;
        if (F->owner[u] >= 0 && cls_find(F->parent, F->owner[u]) == c) continue;
        int st = heap_push(&F->heap[c], F->Od[u], u);
        if (st) return st;
    }
    return ORC_OK;
}

/* Runs class *pc for at most `budget` pops (budget < 0: unlimited).
 * Returns 0 when the class waits at a saddle (its task ends), 1 when the
 * budget ran out (the task goes back to the queue), or an error. */
static int flood_run(flood_t* F, int32_t* pc, int64_t budget) {
    int32_t c = *pc;
    for (;;) {
        if (budget == 0) { *pc = c; return 1; }
        if (budget > 0) --budget;
        if (F->heap[c].n == 0) return -ORC_ERR_INTERNAL;
        hitem it = heap_pop(&F->heap[c]);
        int32_t v = it.v;
        if (F->owner[v] >= 0 && cls_find(F->parent, F->owner[v]) == c) continue;
        if (F->owner[v] < 0) F->owner[v] = c;
        int32_t nb[14];
        int kn = nbrs(F->G, v, nb);
        int h = 0, k = 0;
        for (int j = 0; j < kn; ++j) {
            int32_t u = nb[j];
            if (F->Od[u] <= F->Od[v]) continue;
            ++h;
            if (F->owner[u] >= 0 && cls_find(F->parent, F->owner[u]) == c) ++k;
        }
        if (k == h) {                       /* regular for this propagation */
            int st = push_lower_not_in(F, v, c);
            if (st) return -st;
            continue;
        }
        /* arrival at the saddle v */
        if (F->cnt[v] < 0) F->cnt[v] = h;
        F->cnt[v] -= k;
        F->wait_next[c] = F->wait_head[v];
        F->wait_head[v] = c;
        if (F->cnt[v] > 0) { *pc = c; return 0; }   /* a higher neighbour is still unvisited: stop */
        /* last arrival: merge all propagations stopped here, meld their queues */
        int32_t root = c;
        for (int32_t w = F->wait_head[v]; w >= 0; w = F->wait_next[w]) {
            if (w == root) continue;
            int32_t a = cls_find(F->parent, w), b = cls_find(F->parent, root);
            if (a == b) continue;
            /* the class with the larger queue absorbs the other */
            if (F->heap[a].n > F->heap[b].n) { int32_t t = a; a = b; b = t; }
            int st = heap_meld(&F->heap[b], &F->heap[a]);
            if (st) return -st;
            F->parent[a] = b;
            root = b;
        }
        F->wait_head[v] = -1;
        c = cls_find(F->parent, root);
        int st = push_lower_not_in(F, v, c);
        if (st) return -st;
    }
}

typedef struct { int32_t saddle, top; int64_t key_s, key_t; int32_t cls; } reg_t;

static int cmp_reg(const void* pa, const void* pb) {
    const reg_t* a = (const reg_t*)pa;
    const reg_t* b = (const reg_t*)pb;
    if (a->key_s != b->key_s) return a->key_s < b->key_s ? -1 : 1;
    if (a->key_t != b->key_t) return a->key_t < b->key_t ? -1 : 1;
    return 0;
}

static int auth_has_protected(const grid_t* G, const int32_t* Od, const uint8_t* auth,
                              int64_t* n_unauth) {
    int any = 0;
    int64_t cntu = 0;
    for (int64_t v = 0; v < G->n; ++v) {
        int32_t nb[14];
        int k = nbrs(G, v, nb), ismax = 1;
        for (int j = 0; j < k; ++j) if (Od[nb[j]] > Od[v]) { ismax = 0; break; }
        if (!ismax) continue;
        if (auth[v]) any = 1; else ++cntu;
    }
    *n_unauth = cntu;
    return any;
}

static int regions_flood(const grid_t* G, const int32_t* Od, const uint8_t* auth, uint64_t seed,
                         int32_t* region_of, int32_t* reg_saddle, int32_t* reg_top, int64_t* nreg_out) {
    int64_t n = G->n;
    /* unauthorized maxima, by decreasing order */
    int64_t nu = 0;
    int32_t* U = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * n);
    if (!U || !perm) { free(U); free(perm); return ORC_ERR_OOM; }
    for (int64_t v = 0; v < n; ++v) perm[Od[v]] = (int32_t)v;
    for (int64_t i = n - 1; i >= 0; --i) {
        int32_t v = perm[i];
        int32_t nb[14];
        int k = nbrs(G, v, nb), ismax = 1;
        for (int j = 0; j < k; ++j) if (Od[nb[j]] > Od[v]) { ismax = 0; break; }
        if (ismax && !auth[v]) U[nu++] = v;
    }
    free(perm);
    for (int64_t v = 0; v < n; ++v) region_of[v] = -1;
    if (nu == 0) { free(U); *nreg_out = 0; return ORC_OK; }
    int64_t dummy;
    if (!auth_has_protected(G, Od, auth, &dummy)) { free(U); return ORC_ERR_NO_AUTHORIZED; }

    flood_t F;
    F.G = G; F.Od = Od;
    F.owner = (int32_t*)malloc(sizeof(int32_t) * n);
    F.cnt = (int32_t*)malloc(sizeof(int32_t) * n);
    F.wait_head = (int32_t*)malloc(sizeof(int32_t) * n);
    F.wait_next = (int32_t*)malloc(sizeof(int32_t) * nu);
    F.parent = (int32_t*)malloc(sizeof(int32_t) * nu);
    F.heap = (heap_t*)calloc((size_t)nu, sizeof(heap_t));
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (nu + 1));
    int st = ORC_OK;
    if (!F.owner || !F.cnt || !F.wait_head || !F.wait_next || !F.parent || !F.heap || !queue) {
        st = ORC_ERR_OOM; goto done;
    }
    for (int64_t v = 0; v < n; ++v) { F.owner[v] = -1; F.cnt[v] = -1; F.wait_head[v] = -1; }
    for (int64_t c = 0; c < nu; ++c) {
        F.parent[c] = (int32_t)c; F.wait_next[c] = -1;
        st = heap_push(&F.heap[c], Od[U[c]], U[c]);
        if (st) goto done;
    }
    /* task queue: initially every class, in decreasing order of its maximum, or shuffled */
    for (int64_t c = 0; c < nu; ++c) queue[c] = (int32_t)c;
    uint64_t rs = seed;
    if (seed) {
        for (int64_t i = nu - 1; i > 0; --i) {
            int64_t j = (int64_t)(sm64(&rs) % (uint64_t)(i + 1));
            int32_t t = queue[i]; queue[i] = queue[j]; queue[j] = t;
        }
    }
    /* circular task queue; with a seed each task runs for a random slice */
    int64_t qh = 0, qn = nu, qcap = nu + 1;
    int32_t* q2 = (int32_t*)malloc(sizeof(int32_t) * qcap);
    if (!q2) { st = ORC_ERR_OOM; goto done; }
    for (int64_t i = 0; i < nu; ++i) q2[i] = queue[i];
    while (qn > 0) {
        int32_t c = q2[qh]; qh = (qh + 1) % qcap; --qn;
        int64_t budget = seed ? (int64_t)(1 + sm64(&rs) % 7) : -1;
        int r = flood_run(&F, &c, budget);
        if (r < 0) { st = -r; free(q2); goto done; }
        if (r == 1) { q2[(qh + qn) % qcap] = c; ++qn; }
    }
    free(q2);

    /* final stops: every class still waiting at a saddle gives one region */
    {
        reg_t* R = (reg_t*)malloc(sizeof(reg_t) * nu);
        int32_t* cls2reg = (int32_t*)malloc(sizeof(int32_t) * nu);
        int32_t* topv = (int32_t*)malloc(sizeof(int32_t) * nu);
        if (!R || !cls2reg || !topv) { free(R); free(cls2reg); free(topv); st = ORC_ERR_OOM; goto done; }
        for (int64_t c = 0; c < nu; ++c) { cls2reg[c] = -1; topv[c] = -1; }
        /* top of each class: its highest member */
        for (int64_t v = 0; v < n; ++v) {
            if (F.owner[v] < 0 || F.wait_head[v] >= 0) continue;
            int32_t c = cls_find(F.parent, F.owner[v]);
            if (topv[c] < 0 || Od[v] > Od[topv[c]]) topv[c] = (int32_t)v;
        }
        int64_t nr = 0;
        for (int64_t v = 0; v < n; ++v) {
            for (int32_t w = F.wait_head[v]; w >= 0; w = F.wait_next[w]) {
                if (F.cnt[v] <= 0 || cls_find(F.parent, w) != w) { st = ORC_ERR_INTERNAL; break; }
                R[nr].saddle = (int32_t)v; R[nr].top = topv[w]; R[nr].cls = w;
                R[nr].key_s = Od[v]; R[nr].key_t = Od[topv[w]];
                ++nr;
            }
        }
        if (!st) {
            qsort(R, (size_t)nr, sizeof(reg_t), cmp_reg);
            for (int64_t r = 0; r < nr; ++r) {
                cls2reg[R[r].cls] = (int32_t)r;
                reg_saddle[r] = R[r].saddle; reg_top[r] = R[r].top;
            }
            for (int64_t v = 0; v < n; ++v) {
                if (F.owner[v] < 0 || F.wait_head[v] >= 0) continue;
                int32_t c = cls_find(F.parent, F.owner[v]);
                if (cls2reg[c] < 0) { st = ORC_ERR_INTERNAL; break; }
                region_of[v] = cls2reg[c];
            }
            *nreg_out = nr;
        }
        free(R); free(cls2reg); free(topv);
    }

done:
    if (F.heap) for (int64_t c = 0; c < nu; ++c) heap_free(&F.heap[c]);
    free(F.owner); free(F.cnt); free(F.wait_head); free(F.wait_next); free(F.parent);
    free(F.heap); free(queue); free(U);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Persistence-driven selection by propagations (Sec. 4.5): step 1 started  */
/* from every maximum of Od.  Each class keeps its highest maximum m (the    */
/* oldest of the classes it absorbed) and, at every pop of a vertex v, the   */
/* scalar difference between m and v: f(m) - f(v) in the maxima pass,       */
/* f(v) - f(m) in the minima pass, in double precision.  Once it exceeds     */
/* eps the propagation ends and m is persistent.  A class whose queue runs   */
/* dry has covered the whole grid: its maximum is the global one, which is   */
/* kept as well.  Every other maximum ends inside a class that merged into   */
/* an older one, or that waits for ever at a saddle: it is not persistent.   */
/* ------------------------------------------------------------------------ */

static int pers_flood_run(flood_t* F, const float* f, int dir, double eps, int32_t* top,
                          uint8_t* persistent, int32_t* pc, int64_t budget) {
    int32_t c = *pc;
    for (;;) {
        if (budget == 0) { *pc = c; return 1; }
        if (budget > 0) --budget;
        if (F->heap[c].n == 0) { persistent[top[c]] = 1; return 0; }
        hitem it = heap_pop(&F->heap[c]);
        int32_t v = it.v;
        if (F->owner[v] >= 0 && cls_find(F->parent, F->owner[v]) == c) continue;
        double d = dir > 0 ? (double)f[top[c]] - (double)f[v] : (double)f[v] - (double)f[top[c]];
        if (d > eps) { persistent[top[c]] = 1; return 0; }
        if (F->owner[v] < 0) F->owner[v] = c;
        int32_t nb[14];
        int kn = nbrs(F->G, v, nb);
        int h = 0, k = 0;
        for (int j = 0; j < kn; ++j) {
            int32_t u = nb[j];
            if (F->Od[u] <= F->Od[v]) continue;
            ++h;
            if (F->owner[u] >= 0 && cls_find(F->parent, F->owner[u]) == c) ++k;
        }
        if (k == h) {
            int st = push_lower_not_in(F, v, c);
            if (st) return -st;
            continue;
        }
        if (F->cnt[v] < 0) F->cnt[v] = h;
        F->cnt[v] -= k;
        F->wait_next[c] = F->wait_head[v];
        F->wait_head[v] = c;
        if (F->cnt[v] > 0) { *pc = c; return 0; }
        int32_t root = c;
        for (int32_t w = F->wait_head[v]; w >= 0; w = F->wait_next[w]) {
            if (w == root) continue;
            int32_t a = cls_find(F->parent, w), b = cls_find(F->parent, root);
            if (a == b) continue;
            if (F->heap[a].n > F->heap[b].n) { int32_t t = a; a = b; b = t; }
            int st = heap_meld(&F->heap[b], &F->heap[a]);
            if (st) return -st;
            F->parent[a] = b;
            if (F->Od[top[a]] > F->Od[top[b]]) top[b] = top[a];   /* the elder survives */
            root = b;
        }
        F->wait_head[v] = -1;
        c = cls_find(F->parent, root);
        int st = push_lower_not_in(F, v, c);
        if (st) return -st;
    }
}

static int pers_select(const grid_t* G, const float* f, const int32_t* O, int dir, double eps, uint64_t seed,
                       uint8_t* persistent) {
    int64_t n = G->n;
    int st = ORC_OK;
    int64_t nu = 0;
    int32_t* Od = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* U = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * n);
    flood_t F;
    memset(&F, 0, sizeof F);
    int32_t* top = NULL;
    int32_t* q2 = NULL;
    if (!Od || !U || !perm) { st = ORC_ERR_OOM; goto done; }
    for (int64_t v = 0; v < n; ++v) {
        Od[v] = dir > 0 ? O[v] : (int32_t)(n - 1 - O[v]);
        persistent[v] = 0;
    }
    for (int64_t v = 0; v < n; ++v) perm[Od[v]] = (int32_t)v;
    for (int64_t i = n - 1; i >= 0; --i) {             /* every maximum of Od, highest first */
        int32_t v = perm[i];
        int32_t nb[14];
        int k = nbrs(G, v, nb), ismax = 1;
        for (int j = 0; j < k; ++j) if (Od[nb[j]] > Od[v]) { ismax = 0; break; }
        if (ismax) U[nu++] = v;
    }
    F.G = G; F.Od = Od;
    F.owner = (int32_t*)malloc(sizeof(int32_t) * n);
    F.cnt = (int32_t*)malloc(sizeof(int32_t) * n);
    F.wait_head = (int32_t*)malloc(sizeof(int32_t) * n);
    F.wait_next = (int32_t*)malloc(sizeof(int32_t) * nu);
    F.parent = (int32_t*)malloc(sizeof(int32_t) * nu);
    F.heap = (heap_t*)calloc((size_t)nu, sizeof(heap_t));
    top = (int32_t*)malloc(sizeof(int32_t) * nu);
    q2 = (int32_t*)malloc(sizeof(int32_t) * (nu + 1));
    if (!F.owner || !F.cnt || !F.wait_head || !F.wait_next || !F.parent || !F.heap || !top || !q2) {
        st = ORC_ERR_OOM; goto done;
    }
    for (int64_t v = 0; v < n; ++v) { F.owner[v] = -1; F.cnt[v] = -1; F.wait_head[v] = -1; }
    for (int64_t c = 0; c < nu; ++c) {
        F.parent[c] = (int32_t)c; F.wait_next[c] = -1; top[c] = U[c];
        st = heap_push(&F.heap[c], Od[U[c]], U[c]);
        if (st) goto done;
        q2[c] = (int32_t)c;
    }
    uint64_t rs = seed;
    if (seed) {
        for (int64_t i = nu - 1; i > 0; --i) {
            int64_t j = (int64_t)(sm64(&rs) % (uint64_t)(i + 1));
            int32_t t = q2[i]; q2[i] = q2[j]; q2[j] = t;
        }
    }
    {
        int64_t qh = 0, qn = nu, qcap = nu + 1;
        while (qn > 0) {
            int32_t c = q2[qh]; qh = (qh + 1) % qcap; --qn;
            int64_t budget = seed ? (int64_t)(1 + sm64(&rs) % 7) : -1;
            int r = pers_flood_run(&F, f, dir, eps, top, persistent, &c, budget);
            if (r < 0) { st = -r; goto done; }
            if (r == 1) { q2[(qh + qn) % qcap] = c; ++qn; }
        }
    }
done:
    if (F.heap) for (int64_t c = 0; c < nu; ++c) heap_free(&F.heap[c]);
    free(F.owner); free(F.cnt); free(F.wait_head); free(F.wait_next); free(F.parent); free(F.heap);
    free(top); free(q2); free(Od); free(U); free(perm);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Step 1, method B: a global join-tree sweep (superlevel set components by  */
/* decreasing order, union-find over vertices).  A component is protected    */
/* when it holds an authorized maximum.  At a vertex whose higher neighbours */
/* lie in several components, at least one protected, every unprotected one */
/* D yields the region D + {v}.  Used to cross-check method A.               */
/* ------------------------------------------------------------------------ */

static int regions_jointree(const grid_t* G, const int32_t* Od, const uint8_t* auth,
                            int32_t* region_of, int32_t* reg_saddle, int32_t* reg_top, int64_t* nreg_out) {
    int64_t n = G->n;
    int64_t* par = (int64_t*)malloc(sizeof(int64_t) * n);
    uint8_t* prot = (uint8_t*)malloc(n);
    int32_t* head = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* tail = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* next = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* top = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * n);
    reg_t* R = NULL;
    int64_t nr = 0, rcap = 0;
    int st = ORC_OK;
    if (!par || !prot || !head || !tail || !next || !top || !perm) { st = ORC_ERR_OOM; goto out; }
    for (int64_t v = 0; v < n; ++v) { par[v] = -1; perm[Od[v]] = (int32_t)v; region_of[v] = -1; }
    int64_t nunauth = 0;
    int anyprot = auth_has_protected(G, Od, auth, &nunauth);
    if (nunauth > 0 && !anyprot) { st = ORC_ERR_NO_AUTHORIZED; goto out; }
    for (int64_t i = n - 1; i >= 0; --i) {
        int32_t v = perm[i];
        int32_t nb[14];
        int k = nbrs(G, v, nb);
        int64_t roots[14]; int nroot = 0;
        for (int j = 0; j < k; ++j) {
            if (Od[nb[j]] <= Od[v]) continue;
            int64_t r = uf_find64(par, nb[j]);
            int dup = 0;
            for (int q = 0; q < nroot; ++q) if (roots[q] == r) dup = 1;
            if (!dup) roots[nroot++] = r;
        }
        par[v] = v; head[v] = v; tail[v] = v; next[v] = -1; top[v] = v;
        if (nroot == 0) { prot[v] = auth[v] ? 1 : 0; continue; }
        int any = 0;
        for (int q = 0; q < nroot; ++q) any |= prot[roots[q]];
        if (nroot >= 2 && any) {
            for (int q = 0; q < nroot; ++q) {
                int64_t r = roots[q];
                if (prot[r]) continue;
                if (nr == rcap) {
                    rcap = rcap ? 2 * rcap : 64;
                    reg_t* nR = (reg_t*)realloc(R, sizeof(reg_t) * rcap);
                    if (!nR) { st = ORC_ERR_OOM; goto out; }
                    R = nR;
                }
                R[nr].saddle = v; R[nr].top = top[r]; R[nr].key_s = Od[v]; R[nr].key_t = Od[top[r]];
                R[nr].cls = (int32_t)nr;
                for (int32_t u = head[r]; u >= 0; u = next[u]) region_of[u] = (int32_t)nr;
                ++nr;
            }
        }
        /* merge every component and v; the merged component is protected if any part was */
        int64_t keep = roots[0];
        for (int q = 1; q < nroot; ++q) {
            int64_t r = roots[q];
            par[r] = keep;
            next[tail[keep]] = head[r];
            tail[keep] = tail[r];
            if (Od[top[r]] > Od[top[keep]]) top[keep] = top[r];
        }
        par[v] = keep;
        next[tail[keep]] = v; tail[keep] = v;
        prot[keep] = (uint8_t)any;
    }
    /* canonical numbering */
    if (nr > 0) {
        int32_t* remap = (int32_t*)malloc(sizeof(int32_t) * nr);
        if (!remap) { st = ORC_ERR_OOM; goto out; }
        qsort(R, (size_t)nr, sizeof(reg_t), cmp_reg);
        for (int64_t r = 0; r < nr; ++r) { remap[R[r].cls] = (int32_t)r; reg_saddle[r] = R[r].saddle; reg_top[r] = R[r].top; }
        for (int64_t v = 0; v < n; ++v) if (region_of[v] >= 0) region_of[v] = remap[region_of[v]];
        free(remap);
    }
    *nreg_out = nr;
out:
    free(par); free(prot); free(head); free(tail); free(next); free(top); free(perm); free(R);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Step 2 (Sec. 4.2, Eq. 3-5): local order of one region R with saddle s.    */
/*   l0 = Od on R, l0(s) = +inf, l0(a) = -inf for the boundary-adjacent       */
/*   vertex a != s of lowest order whose removal keeps R connected.  Then     */
/*   alternate, as the paper does:                                            */
/*   - a superlevel set propagation from s, the only authorized maximum       */
/*     (largest first); the inverse of the visiting order is the new order;  */
/*   - if some minimum of it has no neighbour outside R, a sublevel set      */
/*     propagation from all current authorized minima: the minima of the     */
/*     current order that have a neighbour outside R (smallest first); the   */
/*     visiting order is the new order;                                      */
/*   until only authorized extrema remain.  Propagations use only edges      */
/*   inside R.  lhat gets values 0..|R|-1 with s at |R|-1.                    */
/*                                                                            */
/*   Taken literally the alternation can cycle for ever (a cluster hanging   */
/*   off a cut vertex of R swaps a stray minimum and maximum at every        */
/*   iteration).  So: if the literal alternation has not ended after         */
/*   2|R|+2 propagations, or has no authorized minimum to start from, the    */
/*   region is redone from the first propagation's order with every vertex  */
/*   allowed to be a minimum (all of R\{s} with an outside neighbour) as the */
/*   seeds of each sublevel propagation.  A repeated order after a           */
/*   superlevel propagation proves a cycle; it is detected with Brent's      */
/*   method (one saved order) and only ends the literal attempt early: the  */
/*   result is the same as with the cap alone.                               */
/* ------------------------------------------------------------------------ */

#define ORC_LO_ADOPTED 0      /* literal alternation, all-boundary seeding if it does not end */
#define ORC_LO_LITERAL 1      /* literal alternation only (ORC_ERR_CYCLE if it does not end) */
#define ORC_LO_BOUNDARY 2     /* all-boundary seeding only */
#define ORC_ERR_CYCLE 8

typedef struct {
    const grid_t* G;
    const int32_t* Od;
    int32_t* loc;   /* vertex -> local index in the current region, -1 elsewhere */
} lo_ctx;

/* Articulation points of the graph induced on R (Tarjan's lowpoint method,
 * iterative depth-first search from `root`): is_cut[i] = 1 when removing
 * vertex i disconnects the rest of R. */
static int cut_vertices(const int32_t* adj, const int8_t* deg, int32_t r, int32_t root, uint8_t* is_cut) {
    int32_t* disc = (int32_t*)malloc(sizeof(int32_t) * (size_t)r);
    int32_t* low = (int32_t*)malloc(sizeof(int32_t) * (size_t)r);
    int32_t* par = (int32_t*)malloc(sizeof(int32_t) * (size_t)r);
    int8_t* it = (int8_t*)malloc((size_t)r);
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)r);
    if (!disc || !low || !par || !it || !stack) {
        free(disc); free(low); free(par); free(it); free(stack);
        return ORC_ERR_OOM;
    }
    for (int32_t i = 0; i < r; ++i) { disc[i] = -1; is_cut[i] = 0; it[i] = 0; par[i] = -1; }
    int32_t t = 0, sp = 0, root_children = 0;
    disc[root] = low[root] = t++;
    stack[sp++] = root;
    while (sp > 0) {
        int32_t u = stack[sp - 1];
        if (it[u] < deg[u]) {
            int32_t w = adj[14 * (size_t)u + it[u]++];
            if (disc[w] < 0) {
                par[w] = u;
                disc[w] = low[w] = t++;
                stack[sp++] = w;
                if (u == root) ++root_children;
            } else if (w != par[u] && disc[w] < low[u]) {
                low[u] = disc[w];
            }
        } else {
            --sp;
            int32_t p = par[u];
            if (p >= 0) {
                if (low[u] < low[p]) low[p] = low[u];
                if (p != root && low[u] >= disc[p]) is_cut[p] = 1;
            }
        }
    }
    if (root_children > 1) is_cut[root] = 1;
    free(disc); free(low); free(par); free(it); free(stack);
    return ORC_OK;
}

/* The region's induced graph and the orders of one local simplification. */
typedef struct {
    int32_t r, sidx;
    int32_t* adj;       /* 14 slots per vertex: local indices of neighbours inside R */
    int8_t* deg;
    uint8_t* bnd;       /* has a neighbour outside R */
    uint8_t* seed;      /* seeds of a sublevel set propagation */
    uint8_t* vis;
    int64_t* L2;        /* output of a propagation */
    heap_t H;
} lo_region;

/* Superlevel set propagation from s by the order L (largest first):
 * L[q_i] := r-1-i for the i-th visited vertex q_i. */
static int lo_max_flood(lo_region* Q, int64_t* L) {
    int32_t r = Q->r;
    memset(Q->vis, 0, (size_t)r);
    Q->H.n = 0;
    int st = heap_push(&Q->H, L[Q->sidx], Q->sidx);
    if (st) return st;
    int64_t i = 0;
    while (Q->H.n > 0) {
        hitem it = heap_pop(&Q->H);
        if (Q->vis[it.v]) continue;
        Q->vis[it.v] = 1;
        Q->L2[it.v] = (int64_t)r - 1 - i;
        ++i;
        for (int j = 0; j < Q->deg[it.v]; ++j) {
            int32_t u = Q->adj[14 * (size_t)it.v + j];
            if (!Q->vis[u] && (st = heap_push(&Q->H, L[u], u))) return st;
        }
    }
    if (i != r) return ORC_ERR_INTERNAL;
    memcpy(L, Q->L2, sizeof(int64_t) * (size_t)r);
    return ORC_OK;
}

/* Sublevel set propagation from every vertex with seed[] set (smallest
 * first): L[q_i] := i. */
static int lo_min_flood(lo_region* Q, int64_t* L) {
    int32_t r = Q->r;
    memset(Q->vis, 0, (size_t)r);
    Q->H.n = 0;
    int st;
    for (int32_t u = 0; u < r; ++u)
        if (Q->seed[u] && (st = heap_push(&Q->H, -L[u], u))) return st;
    int64_t i = 0;
    while (Q->H.n > 0) {
        hitem it = heap_pop(&Q->H);
        if (Q->vis[it.v]) continue;
        Q->vis[it.v] = 1;
        Q->L2[it.v] = i;
        ++i;
        for (int j = 0; j < Q->deg[it.v]; ++j) {
            int32_t u = Q->adj[14 * (size_t)it.v + j];
            if (!Q->vis[u] && (st = heap_push(&Q->H, -L[u], u))) return st;
        }
    }
    if (i != r) return ORC_ERR_INTERNAL;
    memcpy(L, Q->L2, sizeof(int64_t) * (size_t)r);
    return ORC_OK;
}

static int lo_is_min(const lo_region* Q, const int64_t* L, int32_t u) {
    for (int j = 0; j < Q->deg[u]; ++j) if (L[Q->adj[14 * (size_t)u + j]] < L[u]) return 0;
    return 1;
}

static int lo_is_max(const lo_region* Q, const int64_t* L, int32_t u) {
    for (int j = 0; j < Q->deg[u]; ++j) if (L[Q->adj[14 * (size_t)u + j]] > L[u]) return 0;
    return 1;
}

/* Unauthorized minima: minima of L without a neighbour outside R. */
static int lo_has_unauth_min(const lo_region* Q, const int64_t* L) {
    for (int32_t u = 0; u < Q->r; ++u) if (!Q->bnd[u] && lo_is_min(Q, L, u)) return 1;
    return 0;
}

/* Unauthorized maxima: maxima of L other than s. */
static int lo_has_unauth_max(const lo_region* Q, const int64_t* L) {
    for (int32_t u = 0; u < Q->r; ++u) if (u != Q->sidx && lo_is_max(Q, L, u)) return 1;
    return 0;
}

/* The alternation from L (the order after the first superlevel set
 * propagation).  literal: sublevel propagations start from the current
 * authorized minima, with Brent's cycle check on the orders after each
 * superlevel propagation (saved: the one order kept for it); otherwise from
 * every vertex allowed to be a minimum.  Returns ORC_OK with L final and
 * *floods the propagations of the whole run (the first one included), or
 * ORC_ERR_CYCLE when the run does not end (cycle, cap or no seed). */
static int lo_alternate(lo_region* Q, int64_t* L, int literal, int64_t* saved, int32_t* floods,
                        int64_t* trace, int32_t max_trace, int32_t* n_trace) {
    int32_t r = Q->r;
    int64_t cap = 2 * (int64_t)r + 2;
    int32_t fl = 1;
    int64_t power = 1, lam = 0;
    int st;
    if (literal) memcpy(saved, L, sizeof(int64_t) * (size_t)r);
    for (;;) {
        if (!lo_has_unauth_min(Q, L)) break;
        int any = 0;
        for (int32_t u = 0; u < r; ++u) {
            Q->seed[u] = (uint8_t)(u != Q->sidx && Q->bnd[u] && (!literal || lo_is_min(Q, L, u)));
            any |= Q->seed[u];
        }
        if (!any) return literal ? ORC_ERR_CYCLE : ORC_ERR_INTERNAL;
        if (++fl > cap) return literal ? ORC_ERR_CYCLE : ORC_ERR_INTERNAL;
        if ((st = lo_min_flood(Q, L))) return st;
        if (trace && *n_trace < max_trace) memcpy(trace + (size_t)(*n_trace)++ * r, L, sizeof(int64_t) * (size_t)r);
        if (!lo_has_unauth_max(Q, L)) break;
        if (++fl > cap) return literal ? ORC_ERR_CYCLE : ORC_ERR_INTERNAL;
        if ((st = lo_max_flood(Q, L))) return st;
        if (trace && *n_trace < max_trace) memcpy(trace + (size_t)(*n_trace)++ * r, L, sizeof(int64_t) * (size_t)r);
        if (literal) {
            if (memcmp(saved, L, sizeof(int64_t) * (size_t)r) == 0) return ORC_ERR_CYCLE;
            if (++lam == power) { memcpy(saved, L, sizeof(int64_t) * (size_t)r); power *= 2; lam = 0; }
        }
    }
    *floods = fl;
    return ORC_OK;
}

/* One region.  rule: ORC_LO_ADOPTED, ORC_LO_LITERAL or ORC_LO_BOUNDARY.
 * *fell_back = 1 when the adopted rule redid the region with all-boundary
 * seeds.  trace (optional): the orders after each propagation, first one
 * included, of the run whose result is returned, max_trace orders at most. */
static int local_order_one(lo_ctx* C, const int32_t* verts, int32_t r, int32_t sidx, int rule,
                           int32_t* lhat_local, int32_t* floods_out, int32_t* fell_back,
                           int64_t* trace, int32_t max_trace, int32_t* n_trace) {
    int st = ORC_OK;
    lo_region Q;
    memset(&Q, 0, sizeof Q);
    Q.r = r; Q.sidx = sidx;
    Q.adj = (int32_t*)malloc(sizeof(int32_t) * 14 * (size_t)r);
    Q.deg = (int8_t*)malloc((size_t)r);
    Q.bnd = (uint8_t*)malloc((size_t)r);
    Q.seed = (uint8_t*)malloc((size_t)r);
    Q.vis = (uint8_t*)malloc((size_t)r);
    Q.L2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)r);
    int64_t* L = (int64_t*)malloc(sizeof(int64_t) * (size_t)r);
    int64_t* L1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)r);
    int64_t* saved = (int64_t*)malloc(sizeof(int64_t) * (size_t)r);
    int32_t nt = 0;
    if (fell_back) *fell_back = 0;
    if (!Q.adj || !Q.deg || !Q.bnd || !Q.seed || !Q.vis || !Q.L2 || !L || !L1 || !saved) { st = ORC_ERR_OOM; goto out; }
    for (int32_t i = 0; i < r; ++i) {
        int32_t nb[14];
        int k = nbrs(C->G, verts[i], nb);
        Q.deg[i] = 0; Q.bnd[i] = 0;
        for (int j = 0; j < k; ++j) {
            int32_t li = C->loc[nb[j]];
            if (li < 0) Q.bnd[i] = 1; else Q.adj[14 * (size_t)i + Q.deg[i]++] = li;
        }
    }
    /* l0.  The vertex set to minus infinity must be visited last by the
     * first superlevel set propagation from s, otherwise it does not end up
     * as a minimum and no authorized minimum is left; this holds exactly when
     * its removal leaves R connected.  Such a boundary-adjacent vertex always
     * exists because the grid graph is 2-connected. */
    if ((st = cut_vertices(Q.adj, Q.deg, r, sidx, Q.vis))) goto out;
    int32_t a = -1;
    for (int32_t i = 0; i < r; ++i) {
        L[i] = C->Od[verts[i]];
        if (i != sidx && Q.bnd[i] && !Q.vis[i] && (a < 0 || C->Od[verts[i]] < C->Od[verts[a]])) a = i;
    }
    if (a < 0) { st = ORC_ERR_INTERNAL; goto out; }
    L[sidx] = INT64_MAX;
    L[a] = INT64_MIN;
    /* first iteration: superlevel set propagation from s */
    if ((st = lo_max_flood(&Q, L))) goto out;
    memcpy(L1, L, sizeof(int64_t) * (size_t)r);
    if (trace && nt < max_trace) memcpy(trace + (size_t)nt++ * r, L, sizeof(int64_t) * (size_t)r);
    st = lo_alternate(&Q, L, rule != ORC_LO_BOUNDARY, saved, floods_out, trace, max_trace, &nt);
    if (st == ORC_ERR_CYCLE && rule == ORC_LO_ADOPTED) {
        if (fell_back) *fell_back = 1;
        memcpy(L, L1, sizeof(int64_t) * (size_t)r);
        nt = trace && max_trace > 0 ? 1 : 0;
        st = lo_alternate(&Q, L, 0, saved, floods_out, trace, max_trace, &nt);
    }
    if (st) goto out;
    for (int32_t u = 0; u < r; ++u) lhat_local[u] = (int32_t)L[u];
out:
    if (n_trace) *n_trace = nt;
    free(Q.adj); free(Q.deg); free(Q.bnd); free(Q.seed); free(Q.vis); free(Q.L2); heap_free(&Q.H);
    free(L); free(L1); free(saved);
    return st;
}

/* Local orders of all regions.  lhat[v] for every member v (saddles keep -1);
 * reg_fallback (optional): 1 for the regions the adopted rule redid. */
static int local_orders(const grid_t* G, const int32_t* Od, const int32_t* region_of,
                        const int32_t* reg_saddle, int64_t nreg, int rule, int32_t* lhat, int32_t* reg_floods,
                        int32_t* reg_fallback) {
    int64_t n = G->n;
    int st = ORC_OK;
    int64_t* start = (int64_t*)calloc((size_t)nreg + 1, sizeof(int64_t));
    int32_t* members = NULL;
    int32_t* loc = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* verts = NULL;
    int32_t* ll = NULL;
    if (!start || !loc) { st = ORC_ERR_OOM; goto out; }
    for (int64_t v = 0; v < n; ++v) { loc[v] = -1; lhat[v] = -1; }
    for (int64_t v = 0; v < n; ++v) if (region_of[v] >= 0) start[region_of[v] + 1]++;
    for (int64_t r = 0; r < nreg; ++r) start[r + 1] += start[r];
    members = (int32_t*)malloc(sizeof(int32_t) * (start[nreg] + 1));
    if (!members) { st = ORC_ERR_OOM; goto out; }
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nreg + 1));
        if (!fill) { st = ORC_ERR_OOM; goto out; }
        memcpy(fill, start, sizeof(int64_t) * ((size_t)nreg + 1));
        for (int64_t v = 0; v < n; ++v) if (region_of[v] >= 0) members[fill[region_of[v]]++] = (int32_t)v;
        free(fill);
    }
    int64_t maxr = 0;
    for (int64_t r = 0; r < nreg; ++r) if (start[r + 1] - start[r] > maxr) maxr = start[r + 1] - start[r];
    verts = (int32_t*)malloc(sizeof(int32_t) * (maxr + 1));
    ll = (int32_t*)malloc(sizeof(int32_t) * (maxr + 1));
    if (!verts || !ll) { st = ORC_ERR_OOM; goto out; }
    lo_ctx C; C.G = G; C.Od = Od; C.loc = loc;
    for (int64_t r = 0; r < nreg; ++r) {
        int32_t m = (int32_t)(start[r + 1] - start[r]);
        for (int32_t i = 0; i < m; ++i) { verts[i] = members[start[r] + i]; loc[verts[i]] = i; }
        verts[m] = reg_saddle[r];
        loc[reg_saddle[r]] = m;
        int32_t fl = 0, fb = 0;
        st = local_order_one(&C, verts, m + 1, m, rule, ll, &fl, &fb, NULL, 0, NULL);
        if (reg_fallback) reg_fallback[r] = fb;
        for (int32_t i = 0; i <= m; ++i) loc[verts[i]] = -1;
        if (st) goto out;
        for (int32_t i = 0; i < m; ++i) lhat[verts[i]] = ll[i];
        reg_floods[r] = fl;
    }
out:
    free(start); free(members); free(loc); free(verts); free(ll);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Optional post-process of step 3 (Sec. 4.2): restoring authorized extrema   */
/* of the other kind that a region swallowed.  In the maxima pass a region R  */
/* can contain authorized minima of the pass's input order; all their         */
/* neighbours lie in R (they are higher than the minimum, hence above s and   */
/* connected to it), and the local order of step 2 makes none of them a       */
/* minimum.  The paper restores such a minimum by making it smaller than all  */
/* its neighbours.  Read here as: the swallowed authorized minima of R are    */
/* taken in increasing order; each one moves below every vertex of the block  */
/* of R (below the ones already restored: they are never adjacent), unless a  */
/* neighbour u of it would then have no higher neighbour left (u would become */
/* a maximum, an unauthorized extremum, breaking Eq. 1); such a minimum stays */
/* swallowed.  Vertices outside R next to a vertex of R other than s are      */
/* below the block of R, so only s and the vertices of R can be higher.       */
/* lhat is renumbered: the restored vertices first, the others in their order.*/
/* Returns the number of restored vertices (added to *restored).              */
/* ------------------------------------------------------------------------ */
static int restore_swallowed(const grid_t* G, const int32_t* Od, const uint8_t* auth, const int32_t* region_of,
                             const int32_t* reg_saddle, int64_t nreg, int32_t* lhat, int64_t* restored) {
    int64_t n = G->n;
    int st = ORC_OK;
    int64_t* key = (int64_t*)malloc(sizeof(int64_t) * n);
    int32_t* cand = NULL;
    int32_t* newr = NULL;
    int64_t* start = (int64_t*)calloc((size_t)nreg + 1, sizeof(int64_t));
    int32_t* members = (int32_t*)malloc(sizeof(int32_t) * (n + 1));
    if (!key || !start || !members) { st = ORC_ERR_OOM; goto out; }
    for (int64_t v = 0; v < n; ++v) if (region_of[v] >= 0) start[region_of[v] + 1]++;
    for (int64_t r = 0; r < nreg; ++r) start[r + 1] += start[r];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nreg + 1));
        if (!fill) { st = ORC_ERR_OOM; goto out; }
        memcpy(fill, start, sizeof(int64_t) * ((size_t)nreg + 1));
        for (int64_t v = 0; v < n; ++v) if (region_of[v] >= 0) members[fill[region_of[v]]++] = (int32_t)v;
        free(fill);
    }
    cand = (int32_t*)malloc(sizeof(int32_t) * (n + 1));
    newr = (int32_t*)malloc(sizeof(int32_t) * (n + 1));
    if (!cand || !newr) { st = ORC_ERR_OOM; goto out; }
    for (int64_t r = 0; r < nreg; ++r) {
        int32_t m = (int32_t)(start[r + 1] - start[r]);
        const int32_t* mem = members + start[r];
        int32_t s = reg_saddle[r];
        /* the swallowed authorized minima of R, in increasing order */
        int32_t k = 0;
        for (int32_t i = 0; i < m; ++i) {
            int32_t w = mem[i];
            if (!auth[w]) continue;
            int32_t nb[14];
            int kn = nbrs(G, w, nb), ismin = 1;
            for (int j = 0; j < kn; ++j) if (Od[nb[j]] < Od[w]) { ismin = 0; break; }
            if (ismin) cand[k++] = w;
        }
        if (k == 0) continue;
        for (int32_t i = 1; i < k; ++i) {             /* insertion sort by Od */
            int32_t w = cand[i], j = i - 1;
            while (j >= 0 && Od[cand[j]] > Od[w]) { cand[j + 1] = cand[j]; --j; }
            cand[j + 1] = w;
        }
        for (int32_t i = 0; i < m; ++i) key[mem[i]] = lhat[mem[i]];
        int32_t done = 0;
        for (int32_t c = 0; c < k; ++c) {
            int32_t w = cand[c];
            int32_t nbw[14];
            int kw = nbrs(G, w, nbw), ok = 1;
            for (int j = 0; j < kw && ok; ++j) {
                int32_t u = nbw[j];
                int32_t nbu[14];
                int ku = nbrs(G, u, nbu), higher = 0;
                for (int t = 0; t < ku && !higher; ++t) {
                    int32_t x = nbu[t];
                    if (x == w) continue;
                    if (x == s) higher = 1;
                    else if (region_of[x] == r && key[x] > key[u]) higher = 1;
                }
                if (!higher) ok = 0;
            }
            if (ok) key[w] = INT64_MIN + done++;     /* below the block, above the earlier restored ones */
        }
        if (done == 0) continue;
        /* renumber: restored first (in the order they were restored), then the
         * others in their order (lhat minus the restored ones below them) */
        for (int32_t i = 0; i < m; ++i) {
            int32_t v = mem[i];
            if (key[v] < 0) continue;
            int32_t below = 0;
            for (int32_t c = 0; c < k; ++c) if (key[cand[c]] < 0 && lhat[cand[c]] < lhat[v]) ++below;
            newr[i] = done + lhat[v] - below;
        }
        for (int32_t i = 0; i < m; ++i) {
            int32_t v = mem[i];
            lhat[v] = key[v] < 0 ? (int32_t)(key[v] - INT64_MIN) : newr[i];
        }
        *restored += done;
    }
out:
    free(key); free(cand); free(newr); free(start); free(members);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Step 3 (Sec. 4.2, Eq. 6): new global order.  Sort key                     */
/*   non-member u (saddles included): (Od(u), 1, 0, 0)                        */
/*   member v of region R:            (Od(s_R), 0, Od(top_R), lhat(v))        */
/* so every region forms a contiguous block right before its saddle, sibling */
/* blocks of one saddle ordered by their highest vertex.                     */
/* Step 4 (zeta = 0): g(v) = g(s_R) for members.                             */
/* ------------------------------------------------------------------------ */

static const int32_t* s_k_od;
static const int32_t* s_k_reg;
static const int32_t* s_k_sad;
static const int32_t* s_k_top;
static const int32_t* s_k_lhat;

static void key_of(int32_t v, int64_t* k) {
    int32_t r = s_k_reg[v];
    if (r < 0) { k[0] = s_k_od[v]; k[1] = 1; k[2] = 0; k[3] = 0; }
    else { k[0] = s_k_od[s_k_sad[r]]; k[1] = 0; k[2] = s_k_od[s_k_top[r]]; k[3] = s_k_lhat[v]; }
}

static int cmp_pair_order(const void* pa, const void* pb) {
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    int64_t ka[4], kb[4];
    key_of(a, ka); key_of(b, kb);
    for (int i = 0; i < 4; ++i) if (ka[i] != kb[i]) return ka[i] < kb[i] ? -1 : 1;
    return 0;
}

/* Values of step 4 (zeta = 0): members take their saddle's value, in
 * float32 (g_in/g_out) or float64 (g_in64/g_out64, when not NULL). */
static int apply_pass(const grid_t* G, const int32_t* Od, const int32_t* region_of,
                      const int32_t* reg_saddle, const int32_t* reg_top, const int32_t* lhat,
                      int32_t* Od_out, const float* g_in, float* g_out, const double* g_in64, double* g_out64) {
    int64_t n = G->n;
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * n);
    if (!idx) return ORC_ERR_OOM;
    for (int64_t v = 0; v < n; ++v) idx[v] = (int32_t)v;
    s_k_od = Od; s_k_reg = region_of; s_k_sad = reg_saddle; s_k_top = reg_top; s_k_lhat = lhat;
    qsort(idx, (size_t)n, sizeof(int32_t), cmp_pair_order);
    for (int64_t i = 0; i < n; ++i) Od_out[idx[i]] = (int32_t)i;
    free(idx);
    for (int64_t v = 0; v < n; ++v) {
        int32_t r = region_of[v];
        if (g_out64) g_out64[v] = (r < 0) ? g_in64[v] : g_in64[reg_saddle[r]];
        else g_out[v] = (r < 0) ? g_in[v] : g_in[reg_saddle[r]];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Public stage entry points (all on the pass-oriented order Od).            */
/* ------------------------------------------------------------------------ */

int orc_regions(int ndim, const int64_t* dims, const int32_t* Od, const uint8_t* auth, int method,
                uint64_t seed, int32_t* region_of, int32_t* reg_saddle, int32_t* reg_top, int64_t* nreg) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    if (method == 0) return regions_flood(&G, Od, auth, seed, region_of, reg_saddle, reg_top, nreg);
    return regions_jointree(&G, Od, auth, region_of, reg_saddle, reg_top, nreg);
}

int orc_local_orders(int ndim, const int64_t* dims, const int32_t* Od, const int32_t* region_of,
                     const int32_t* reg_saddle, int64_t nreg, int32_t* lhat, int32_t* reg_floods) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    return local_orders(&G, Od, region_of, reg_saddle, nreg, ORC_LO_ADOPTED, lhat, reg_floods, NULL);
}

/* Step 2 under a given seeding rule (ORC_LO_*), with the regions redone. */
int orc_local_orders_rule(int ndim, const int64_t* dims, const int32_t* Od, const int32_t* region_of,
                          const int32_t* reg_saddle, int64_t nreg, int rule, int32_t* lhat, int32_t* reg_floods,
                          int32_t* reg_fallback) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    if (rule < ORC_LO_ADOPTED || rule > ORC_LO_BOUNDARY) return ORC_ERR_ARG;
    return local_orders(&G, Od, region_of, reg_saddle, nreg, rule, lhat, reg_floods, reg_fallback);
}

/* Step 2 on one vertex set R (verts[0..r-1], the saddle at verts[sidx]) with
 * the orders after each propagation: trace[i*r + j] is the order of verts[j]
 * after propagation i (at most max_trace of them, *n_trace written). */
int orc_local_order_trace(int ndim, const int64_t* dims, const int32_t* Od, const int32_t* verts, int32_t r,
                          int32_t sidx, int rule, int32_t* lhat_local, int32_t* floods, int32_t* fell_back,
                          int64_t* trace, int32_t max_trace, int32_t* n_trace) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    if (r < 2 || sidx < 0 || sidx >= r || rule < ORC_LO_ADOPTED || rule > ORC_LO_BOUNDARY) return ORC_ERR_ARG;
    int32_t* loc = (int32_t*)malloc(sizeof(int32_t) * G.n);
    if (!loc) return ORC_ERR_OOM;
    for (int64_t v = 0; v < G.n; ++v) loc[v] = -1;
    for (int32_t i = 0; i < r; ++i) {
        if (verts[i] < 0 || verts[i] >= G.n || loc[verts[i]] >= 0) { free(loc); return ORC_ERR_ARG; }
        loc[verts[i]] = i;
    }
    lo_ctx C; C.G = &G; C.Od = Od; C.loc = loc;
    st = local_order_one(&C, verts, r, sidx, rule, lhat_local, floods, fell_back, trace, max_trace, n_trace);
    free(loc);
    return st;
}

int orc_apply(int ndim, const int64_t* dims, const int32_t* Od, const int32_t* region_of,
              const int32_t* reg_saddle, const int32_t* reg_top, const int32_t* lhat,
              const float* g_in, int32_t* Od_out, float* g_out) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    return apply_pass(&G, Od, region_of, reg_saddle, reg_top, lhat, Od_out, g_in, g_out, NULL, NULL);
}

/* One pass on (g, O).  dir = +1: maxima pass; dir = -1: minima pass, run as a
 * maxima pass on the mirrored order N-1-O and mirrored back (Sec. 4:
 * minima are processed symmetrically). */
static int one_pass(const grid_t* G, int dir, const uint8_t* auth, int method, uint64_t seed, int rule,
                    int restore, float* g, double* g64, int32_t* O, orc_stats* S) {
    int64_t n = G->n;
    int st = ORC_OK;
    int32_t* Od = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* region_of = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* reg_saddle = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* reg_top = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* lhat = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* reg_floods = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* reg_fb = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* Od2 = (int32_t*)malloc(sizeof(int32_t) * n);
    float* g2 = g64 ? NULL : (float*)malloc(sizeof(float) * n);
    double* g2d = g64 ? (double*)malloc(sizeof(double) * n) : NULL;
    int64_t nreg = 0;
    int side = dir > 0 ? 1 : 0;
    if (!Od || !region_of || !reg_saddle || !reg_top || !lhat || !reg_floods || !reg_fb || !Od2 || (!g2 && !g2d)) {
        st = ORC_ERR_OOM; goto out;
    }
    for (int64_t v = 0; v < n; ++v) Od[v] = dir > 0 ? O[v] : (int32_t)(n - 1 - O[v]);
    {
        int64_t nun = 0;
        auth_has_protected(G, Od, auth, &nun);
        if (S) S->removed[side] = nun;
    }
    st = method == 0 ? regions_flood(G, Od, auth, seed, region_of, reg_saddle, reg_top, &nreg)
                     : regions_jointree(G, Od, auth, region_of, reg_saddle, reg_top, &nreg);
    if (st) goto out;
    st = local_orders(G, Od, region_of, reg_saddle, nreg, rule, lhat, reg_floods, reg_fb);
    if (st) goto out;
    if (restore) {
        int64_t nres = 0;
        st = restore_swallowed(G, Od, auth, region_of, reg_saddle, nreg, lhat, &nres);
        if (st) goto out;
        if (S) S->restored[side] = nres;
    }
    st = apply_pass(G, Od, region_of, reg_saddle, reg_top, lhat, Od2, g, g2, g64, g2d);
    if (st) goto out;
    for (int64_t v = 0; v < n; ++v) {
        O[v] = dir > 0 ? Od2[v] : (int32_t)(n - 1 - Od2[v]);
        if (g64) g64[v] = g2d[v];
        else g[v] = g2[v];
    }
    if (S) {
        int64_t mem = 0, maxr = 0;
        int32_t mf = 0; int64_t tf = 0, nfb = 0;
        int64_t* sz = (int64_t*)calloc((size_t)nreg + 1, sizeof(int64_t));
        if (!sz) { st = ORC_ERR_OOM; goto out; }
        for (int64_t v = 0; v < n; ++v) if (region_of[v] >= 0) { ++mem; ++sz[region_of[v]]; }
        for (int64_t r = 0; r < nreg; ++r) {
            if (sz[r] > maxr) maxr = sz[r];
            if (reg_floods[r] > mf) mf = reg_floods[r];
            tf += reg_floods[r];
            nfb += reg_fb[r];
        }
        free(sz);
        S->regions[side] = nreg; S->region_vertices[side] = mem; S->max_region[side] = maxr;
        S->max_local_floods[side] = mf; S->total_local_floods[side] = tf; S->fallback_regions[side] = nfb;
    }
out:
    free(Od); free(region_of); free(reg_saddle); free(reg_top); free(lhat); free(reg_floods); free(reg_fb);
    free(Od2); free(g2); free(g2d);
    return st;
}

/* Full LTS: O = order field of f, g = f; then the minima pass and/or the
 * maxima pass.  auth_ids lists the authorized extrema (minima and maxima
 * together; an id that is not an extremum of a pass's kind is ignored by
 * that pass; duplicates are allowed). */
static int lts_rule(int ndim, const int64_t* dims, const float* f, const int32_t* auth_ids, int64_t n_auth,
                    int mode, float* g, int32_t* O, orc_stats* S, int method, uint64_t seed, int rule) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    if ((mode & ~ORC_MODE_RESTORE) < ORC_MODE_MIN || (mode & ~ORC_MODE_RESTORE) > ORC_MODE_BOTH) return ORC_ERR_ARG;
    if (n_auth < 0 || (n_auth > 0 && !auth_ids)) return ORC_ERR_ARG;
    for (int64_t i = 0; i < n_auth; ++i)
        if (auth_ids[i] < 0 || auth_ids[i] >= G.n) return ORC_ERR_ARG;
    if (S) { memset(S, 0, sizeof *S); S->n_vertices = G.n; }
    st = orc_order_field(ndim, dims, f, O);
    if (st) return st;
    uint8_t* auth = (uint8_t*)calloc((size_t)G.n, 1);
    if (!auth) return ORC_ERR_OOM;
    for (int64_t i = 0; i < n_auth; ++i) auth[auth_ids[i]] = 1;
    memcpy(g, f, sizeof(float) * G.n);
    const int restore = (mode & ORC_MODE_RESTORE) != 0;
    if (mode & ORC_MODE_MIN) st = one_pass(&G, -1, auth, method, seed, rule, restore, g, NULL, O, S);
    if (!st && (mode & ORC_MODE_MAX)) st = one_pass(&G, +1, auth, method, seed, rule, restore, g, NULL, O, S);
    free(auth);
    return st;
}

int orc_lts(int ndim, const int64_t* dims, const float* f, const int32_t* auth_ids, int64_t n_auth,
            int mode, float* g, int32_t* O, orc_stats* S, int method, uint64_t seed) {
    return lts_rule(ndim, dims, f, auth_ids, n_auth, mode, g, O, S, method, seed, ORC_LO_ADOPTED);
}

/* The whole method on a float64 field: the order field sorts the float64
 * values (ties by vertex id, -0.0 == +0.0, NaN an error) and members take
 * their saddle's float64 value; everything else works on the order field and
 * is the same as for float32. */
int orc_lts_f64(int ndim, const int64_t* dims, const double* f, const int32_t* auth_ids, int64_t n_auth,
                int mode, double* g, int32_t* O, orc_stats* S) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    if ((mode & ~ORC_MODE_RESTORE) < ORC_MODE_MIN || (mode & ~ORC_MODE_RESTORE) > ORC_MODE_BOTH) return ORC_ERR_ARG;
    if (n_auth < 0 || (n_auth > 0 && !auth_ids)) return ORC_ERR_ARG;
    for (int64_t i = 0; i < n_auth; ++i)
        if (auth_ids[i] < 0 || auth_ids[i] >= G.n) return ORC_ERR_ARG;
    if (S) { memset(S, 0, sizeof *S); S->n_vertices = G.n; }
    st = orc_order_field_f64(ndim, dims, f, O);
    if (st) return st;
    uint8_t* auth = (uint8_t*)calloc((size_t)G.n, 1);
    if (!auth) return ORC_ERR_OOM;
    for (int64_t i = 0; i < n_auth; ++i) auth[auth_ids[i]] = 1;
    memcpy(g, f, sizeof(double) * G.n);
    const int restore = (mode & ORC_MODE_RESTORE) != 0;
    if (mode & ORC_MODE_MIN) st = one_pass(&G, -1, auth, 0, 0, ORC_LO_ADOPTED, restore, NULL, g, O, S);
    if (!st && (mode & ORC_MODE_MAX)) st = one_pass(&G, +1, auth, 0, 0, ORC_LO_ADOPTED, restore, NULL, g, O, S);
    free(auth);
    return st;
}

/* The whole method under a given step-2 seeding rule (ORC_LO_*), for tests. */
int orc_lts_rule(int ndim, const int64_t* dims, const float* f, const int32_t* auth_ids, int64_t n_auth,
                 int mode, float* g, int32_t* O, orc_stats* S, int method, uint64_t seed, int rule) {
    if (rule < ORC_LO_ADOPTED || rule > ORC_LO_BOUNDARY) return ORC_ERR_ARG;
    return lts_rule(ndim, dims, f, auth_ids, n_auth, mode, g, O, S, method, seed, rule);
}

/* One pass on a given (g, O), for stage-wise checks. */
int orc_pass(int ndim, const int64_t* dims, int dir, const int32_t* auth_ids, int64_t n_auth,
             float* g, int32_t* O, orc_stats* S, int method, uint64_t seed) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    uint8_t* auth = (uint8_t*)calloc((size_t)G.n, 1);
    if (!auth) return ORC_ERR_OOM;
    for (int64_t i = 0; i < n_auth; ++i) {
        if (auth_ids[i] < 0 || auth_ids[i] >= G.n) { free(auth); return ORC_ERR_ARG; }
        auth[auth_ids[i]] = 1;
    }
    if (S) { memset(S, 0, sizeof *S); S->n_vertices = G.n; }
    st = one_pass(&G, dir, auth, method, seed, ORC_LO_ADOPTED, 0, g, NULL, O, S);
    free(auth);
    return st;
}

/* Persistence-driven selection (Sec. 4.5) on (f, O): persistent[v] = 1 for the
 * maxima (dir = +1) or minima (dir = -1) that the eps-bounded propagations
 * keep.  seed != 0 runs the propagations in a shuffled, sliced schedule. */
int orc_pers_select(int ndim, const int64_t* dims, const float* f, const int32_t* O, int dir, double eps,
                    uint64_t seed, uint8_t* persistent) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    if (dir != 1 && dir != -1) return ORC_ERR_ARG;
    for (int64_t v = 0; v < G.n; ++v)
        if (isnan(f[v])) return ORC_ERR_NAN;
    return pers_select(&G, f, O, dir, eps, seed, persistent);
}

/* ------------------------------------------------------------------------ */
/* Regions read off the eps-bounded propagations (Sec. 4.5).  A check of a   */
/* single-phase formulation, for tests: every merge gives the merged class a */
/* fresh id, so a claim carries the class as it was when the claim was made, */
/* and each absorbed class records the saddle of its merge.  A class node    */
/* whose highest extremum is not persistent, and that waits for ever at a    */
/* saddle or was merged at a saddle into a node whose extremum is            */
/* persistent, is a region of LTS with the persistent extrema authorized:    */
/* its members are the vertices claimed by it and by the nodes merged into   */
/* it, but that saddle.                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    flood_t F;
    int32_t* top;       /* per node: highest extremum */
    int32_t* mparent;   /* per node: the node it was merged into, or -1 */
    int32_t* msad;      /* per node: the saddle of that merge, or -1 */
    int32_t next;       /* next fresh node id */
} pflood_t;

static int pers_flood_run_nodes(pflood_t* P, const float* f, int dir, double eps, uint8_t* persistent,
                                int32_t* pc, int64_t budget) {
    flood_t* F = &P->F;
    int32_t c = *pc;
    for (;;) {
        if (budget == 0) { *pc = c; return 1; }
        if (budget > 0) --budget;
        if (F->heap[c].n == 0) { persistent[P->top[c]] = 1; return 0; }
        hitem it = heap_pop(&F->heap[c]);
        int32_t v = it.v;
        if (F->owner[v] >= 0 && cls_find(F->parent, F->owner[v]) == c) continue;
        int32_t m = P->top[c];
        double d = dir > 0 ? (double)f[m] - (double)f[v] : (double)f[v] - (double)f[m];
        if (d > eps) { persistent[m] = 1; return 0; }
        if (F->owner[v] < 0) F->owner[v] = c;
        int32_t nb[14];
        int kn = nbrs(F->G, v, nb);
        int h = 0, k = 0;
        for (int j = 0; j < kn; ++j) {
            int32_t u = nb[j];
            if (F->Od[u] <= F->Od[v]) continue;
            ++h;
            if (F->owner[u] >= 0 && cls_find(F->parent, F->owner[u]) == c) ++k;
        }
        if (k == h) {
            int st = push_lower_not_in(F, v, c);
            if (st) return -st;
            continue;
        }
        if (F->cnt[v] < 0) F->cnt[v] = h;
        F->cnt[v] -= k;
        F->wait_next[c] = F->wait_head[v];
        F->wait_head[v] = c;
        if (F->cnt[v] > 0) { *pc = c; return 0; }
        /* last arrival: every class waiting at v becomes a child of a fresh node */
        int32_t nid = P->next++;
        F->parent[nid] = nid;
        P->mparent[nid] = -1;
        P->msad[nid] = -1;
        F->wait_next[nid] = -1;
        int32_t best = -1;
        for (int32_t w = F->wait_head[v]; w >= 0; w = F->wait_next[w]) {
            int32_t a = cls_find(F->parent, w);
            if (a == nid) continue;
            int st = heap_meld(&F->heap[nid], &F->heap[a]);
            if (st) return -st;
            F->parent[a] = nid;
            P->mparent[a] = nid;
            P->msad[a] = v;
            if (best < 0 || F->Od[P->top[a]] > F->Od[best]) best = P->top[a];
        }
        P->top[nid] = best;
        F->wait_head[v] = -1;
        c = nid;
        int st = push_lower_not_in(F, v, c);
        if (st) return -st;
    }
}

int orc_pers_regions(int ndim, const int64_t* dims, const float* f, const int32_t* O, int dir, double eps,
                     uint64_t seed, int32_t* region_of, int32_t* reg_saddle, int32_t* reg_top, int64_t* nreg_out) {
    grid_t G;
    int st = grid_init(&G, ndim, dims);
    if (st) return st;
    if (dir != 1 && dir != -1) return ORC_ERR_ARG;
    int64_t n = G.n;
    pflood_t P;
    memset(&P, 0, sizeof P);
    int32_t* Od = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* U = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * n);
    uint8_t* persistent = (uint8_t*)calloc((size_t)n, 1);
    int32_t *q2 = NULL, *wsad = NULL, *regid = NULL;
    reg_t* R = NULL;
    int64_t nu = 0, cap = 0;
    if (!Od || !U || !perm || !persistent) { st = ORC_ERR_OOM; goto done; }
    for (int64_t v = 0; v < n; ++v) Od[v] = dir > 0 ? O[v] : (int32_t)(n - 1 - O[v]);
    for (int64_t v = 0; v < n; ++v) perm[Od[v]] = (int32_t)v;
    for (int64_t i = n - 1; i >= 0; --i) {
        int32_t v = perm[i];
        int32_t nb[14];
        int k = nbrs(&G, v, nb), ismax = 1;
        for (int j = 0; j < k; ++j) if (Od[nb[j]] > Od[v]) { ismax = 0; break; }
        if (ismax) U[nu++] = v;
    }
    cap = 2 * nu + 1;                      /* seeds and one fresh node per merge */
    P.F.G = &G; P.F.Od = Od;
    P.F.owner = (int32_t*)malloc(sizeof(int32_t) * n);
    P.F.cnt = (int32_t*)malloc(sizeof(int32_t) * n);
    P.F.wait_head = (int32_t*)malloc(sizeof(int32_t) * n);
    P.F.wait_next = (int32_t*)malloc(sizeof(int32_t) * cap);
    P.F.parent = (int32_t*)malloc(sizeof(int32_t) * cap);
    P.F.heap = (heap_t*)calloc((size_t)cap, sizeof(heap_t));
    P.top = (int32_t*)malloc(sizeof(int32_t) * cap);
    P.mparent = (int32_t*)malloc(sizeof(int32_t) * cap);
    P.msad = (int32_t*)malloc(sizeof(int32_t) * cap);
    q2 = (int32_t*)malloc(sizeof(int32_t) * (nu + 1));
    wsad = (int32_t*)malloc(sizeof(int32_t) * cap);
    regid = (int32_t*)malloc(sizeof(int32_t) * cap);
    R = (reg_t*)malloc(sizeof(reg_t) * cap);
    if (!P.F.owner || !P.F.cnt || !P.F.wait_head || !P.F.wait_next || !P.F.parent || !P.F.heap || !P.top ||
        !P.mparent || !P.msad || !q2 || !wsad || !regid || !R) { st = ORC_ERR_OOM; goto done; }
    for (int64_t v = 0; v < n; ++v) { P.F.owner[v] = -1; P.F.cnt[v] = -1; P.F.wait_head[v] = -1; }
    for (int64_t c = 0; c < cap; ++c) { P.mparent[c] = -1; P.msad[c] = -1; wsad[c] = -1; regid[c] = -1; }
    for (int64_t c = 0; c < nu; ++c) {
        P.F.parent[c] = (int32_t)c; P.F.wait_next[c] = -1; P.top[c] = U[c];
        st = heap_push(&P.F.heap[c], Od[U[c]], U[c]);
        if (st) goto done;
        q2[c] = (int32_t)c;
    }
    P.next = (int32_t)nu;
    {
        uint64_t rs = seed;
        if (seed) {
            for (int64_t i = nu - 1; i > 0; --i) {
                int64_t j = (int64_t)(sm64(&rs) % (uint64_t)(i + 1));
                int32_t t = q2[i]; q2[i] = q2[j]; q2[j] = t;
            }
        }
        int64_t qh = 0, qn = nu, qcap = nu + 1;
        while (qn > 0) {
            int32_t c = q2[qh]; qh = (qh + 1) % qcap; --qn;
            int64_t budget = seed ? (int64_t)(1 + sm64(&rs) % 7) : -1;
            int r = pers_flood_run_nodes(&P, f, dir, eps, persistent, &c, budget);
            if (r < 0) { st = -r; goto done; }
            if (r == 1) { q2[(qh + qn) % qcap] = c; ++qn; }
        }
    }
    /* classes waiting for ever, and where */
    for (int64_t v = 0; v < n; ++v)
        for (int32_t w = P.F.wait_head[v]; w >= 0; w = P.F.wait_next[w]) wsad[w] = (int32_t)v;
    /* region nodes */
    {
        int64_t nr = 0;
        for (int32_t x = 0; x < P.next; ++x) {
            if (persistent[P.top[x]]) continue;
            int32_t p = P.mparent[x];
            int32_t s = -1;
            if (p >= 0 && persistent[P.top[p]]) s = P.msad[x];
            else if (p < 0) s = wsad[x];
            if (s < 0) continue;
            R[nr].saddle = s; R[nr].top = P.top[x]; R[nr].cls = x;
            R[nr].key_s = Od[s]; R[nr].key_t = Od[P.top[x]];
            ++nr;
        }
        qsort(R, (size_t)nr, sizeof(reg_t), cmp_reg);
        for (int64_t r = 0; r < nr; ++r) {
            regid[R[r].cls] = (int32_t)r;
            reg_saddle[r] = R[r].saddle; reg_top[r] = R[r].top;
        }
        for (int64_t v = 0; v < n; ++v) {
            region_of[v] = -1;
            int32_t y = P.F.owner[v];
            if (y < 0 || persistent[P.top[y]]) continue;
            int32_t z = y;
            while (P.mparent[z] >= 0 && !persistent[P.top[P.mparent[z]]]) z = P.mparent[z];
            if (regid[z] < 0) { st = ORC_ERR_INTERNAL; goto done; }
            if (R[regid[z]].saddle == (int32_t)v) continue;     /* its saddle, not a member */
            region_of[v] = regid[z];
        }
        *nreg_out = nr;
    }
done:
    if (P.F.heap) for (int64_t c = 0; c < cap; ++c) heap_free(&P.F.heap[c]);
    free(P.F.owner); free(P.F.cnt); free(P.F.wait_head); free(P.F.wait_next); free(P.F.parent); free(P.F.heap);
    free(P.top); free(P.mparent); free(P.msad); free(q2); free(wsad); free(regid); free(R);
    free(Od); free(U); free(perm); free(persistent);
    return st;
}
