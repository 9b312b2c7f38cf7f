/*
 * CPU oracle, C core of isovolume tracking (paper Sec. 6.1, Algorithm 1,
 * right column).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite and the benchmark's
 * CPU-baseline leg, never by the product path.  It shares no code with the
 * CUDA path.
 *
 * What it computes, step by step in the paper's order:
 *   * The level set f = c of a time-varying scalar field on the simplicial
 *     spacetime mesh.  Treating the isovalue test as a 1-D vector field
 *     w(u) = f(u) - c (Sec. 6.1), the symbolic perturbation adds a positive
 *     infinitesimal to w at every vertex, so the perturbed sign of vertex u
 *     is "above" (+) iff f(u) >= c and "below" (-) iff f(u) < c; no vertex
 *     lies on the level set and no edge lies in it.
 *   * Edge pass: every 1-simplex of the Kuhn mesh, (v, v + bits(m)) for a
 *     nonempty axis mask m, is tested; it intersects the level set iff its
 *     two vertices have different perturbed signs.
 *   * Cell pass: for every (d)-simplex (a pentachoron in 3D + time, a
 *     tetrahedron in 2D + time) the intersected edges among its vertex pairs
 *     are united; components of the union are the connected pieces of the
 *     isovolume.  The label of a piece is its smallest edge id.
 *
 * Conventions (shared with the Python layer): axes 0..n-1 are space (x
 * fastest), axis n is time; vertex id g = row-major index with x fastest;
 * the edge of base vertex g and mask m (1 <= m < 2^d) has id
 * g * (2^d - 1) + (m - 1).
 */
#include <stdint.h>
#include <stdlib.h>

static void iso_strides(int d, const int64_t *dims, int64_t *stride) {
    stride[0] = 1;
    for (int a = 1; a < d; ++a) stride[a] = stride[a - 1] * dims[a - 1];
}

static void iso_coords(int d, const int64_t *dims, int64_t g, int64_t *c) {
    for (int a = 0; a < d; ++a) {
        c[a] = g % dims[a];
        g /= dims[a];
    }
}

/* 1 iff vertex g + bits(m) lies in the grid (c = coordinates of g) */
static int iso_in(int d, const int64_t *dims, const int64_t *c, int m) {
    for (int a = 0; a < d; ++a)
        if (((m >> a) & 1) && c[a] + 1 >= dims[a]) return 0;
    return 1;
}

static int64_t iso_offset(int d, const int64_t *stride, int m) {
    int64_t o = 0;
    for (int a = 0; a < d; ++a)
        if ((m >> a) & 1) o += stride[a];
    return o;
}

/*
 * Edge pass.  n = spatial dimension (2 or 3), dims = n spatial extents then
 * nt, f = the samples (x fastest), c = isovalue.  Writes the ids of the
 * intersected edges in increasing order to ids[0..cap) and returns how many
 * there are (possibly more than cap).
 */
int64_t oracle_iso_edges(int n, const int64_t *dims, const double *f, double c, int64_t *ids, int64_t cap) {
    const int d = n + 1;
    const int E = (1 << d) - 1;
    int64_t stride[4], co[4];
    iso_strides(d, dims, stride);
    int64_t nv = 1;
    for (int a = 0; a < d; ++a) nv *= dims[a];
    int64_t cnt = 0;
    for (int64_t g = 0; g < nv; ++g) {
        iso_coords(d, dims, g, co);
        const int s0 = f[g] >= c;
        for (int m = 1; m <= E; ++m) {
            if (!iso_in(d, dims, co, m)) continue;
            const int s1 = f[g + iso_offset(d, stride, m)] >= c;
            if (s0 != s1) {
                if (cnt < cap) ids[cnt] = g * E + (m - 1);
                ++cnt;
            }
        }
    }
    return cnt;
}

static int64_t iso_find(const int64_t *ids, int64_t np, int64_t key) {
    int64_t lo = 0, hi = np;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (ids[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < np && ids[lo] == key) ? lo : -1;
}

static int64_t uf_root(int64_t *parent, int64_t x) {
    int64_t r = x;
    while (parent[r] != r) r = parent[r];
    while (parent[x] != r) {
        const int64_t nx = parent[x];
        parent[x] = r;
        x = nx;
    }
    return r;
}

static void uf_join(int64_t *parent, int64_t a, int64_t b) {
    a = uf_root(parent, a);
    b = uf_root(parent, b);
    if (a == b) return;
    if (a < b) parent[b] = a;
    else parent[a] = b;
}

/*
 * Cell pass.  ids[0..np) = the intersected edges in increasing order (from
 * oracle_iso_edges).  Every cell (base g, chain m_1 < ... < m_d = full,
 * i.e. every ordering of the d axes) whose vertices all lie in the grid
 * unites its intersected edges.  labels[i] = smallest id connected to
 * ids[i].  cell_counts (may be NULL): histogram of intersected edges per
 * cell, indexed 0..(d+1)d/2.  Returns 0, or -1 if an intersected edge of a
 * cell is missing from ids.
 */
int oracle_iso_link(int n, const int64_t *dims, const double *f, double c, const int64_t *ids, int64_t np,
                    int64_t *labels, int64_t *cell_counts) {
    const int d = n + 1;
    const int E = (1 << d) - 1;
    int64_t stride[4], co[4];
    iso_strides(d, dims, stride);
    int64_t nv = 1;
    for (int a = 0; a < d; ++a) nv *= dims[a];
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
    if (!parent) return -2;
    for (int64_t i = 0; i < np; ++i) parent[i] = i;
    int rc = 0;
    /* the orderings of the d axes: each gives the chain of one cell type */
    int perm[4];
    int nperm = 1;
    for (int a = 2; a <= d; ++a) nperm *= a;
    for (int64_t g = 0; g < nv && rc == 0; ++g) {
        iso_coords(d, dims, g, co);
        if (!iso_in(d, dims, co, E)) continue;   /* the cube of g must lie in the grid */
        for (int pi = 0; pi < nperm; ++pi) {
            /* pi-th permutation of 0..d-1 (factorial number system) */
            int avail[4] = {0, 1, 2, 3}, na = d, r = pi;
            for (int k = 0; k < d; ++k) {
                int fact = 1;
                for (int q = 2; q <= d - 1 - k; ++q) fact *= q;
                const int j = r / fact;
                r %= fact;
                perm[k] = avail[j];
                for (int q = j; q < na - 1; ++q) avail[q] = avail[q + 1];
                --na;
            }
            int chain[5];
            chain[0] = 0;
            for (int k = 0; k < d; ++k) chain[k + 1] = chain[k] | (1 << perm[k]);
            int above[5];
            for (int k = 0; k <= d; ++k) above[k] = f[g + iso_offset(d, stride, chain[k])] >= c;
            int64_t hit[10];
            int nh = 0;
            for (int i = 0; i <= d; ++i)
                for (int j = i + 1; j <= d; ++j) {
                    if (above[i] == above[j]) continue;
                    const int64_t gb = g + iso_offset(d, stride, chain[i]);
                    const int64_t id = gb * E + ((chain[j] ^ chain[i]) - 1);
                    const int64_t k = iso_find(ids, np, id);
                    if (k < 0) rc = -1;
                    else hit[nh++] = k;
                }
            if (cell_counts) ++cell_counts[nh];
            for (int q = 1; q < nh; ++q) uf_join(parent, hit[0], hit[q]);
        }
    }
    for (int64_t i = 0; i < np; ++i) labels[i] = ids[uf_root(parent, i)];
    free(parent);
    return rc;
}
