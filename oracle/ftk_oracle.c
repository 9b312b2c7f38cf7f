/*
 * CPU oracle, C core: exact puncture predicate with Simulation of Simplicity.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of what the tracking method decides for every n-simplex of the
 * simplicial spacetime mesh.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA
 * path.
 *
 * What it computes (paper Sec. 4.2-4.3):
 *   * An n-simplex (face) with vertices u_0 < ... < u_n (global vertex id)
 *     and integer vectors v_k = G(u_k) in Z^n is punctured iff 0 lies in the
 *     interior of conv(v_0..v_n) (Sec. 4.3, point-in-simplex via the signs of
 *     the determinants of (v_0..v_n, 1)).  By Cramer's rule on Eq. (1) the
 *     barycentric numerators are D_k = (-1)^(n+k) det(V without column k),
 *     so the test is: (-1)^k sign det(V_{-k}) equal for k = 0..n.
 *   * Degenerate determinants are decided by Simulation of Simplicity
 *     (Sec. 2.4, Sec. 4.3): component r of vertex g is perturbed by
 *     eps^(2^(g*n + r)).  Within one determinant the columns are sorted by
 *     vertex id, so entry (row r, column c) carries local key c*n + r and a
 *     set P of perturbed entries has exponent sum_{(r,c) in P} 2^key, i.e.
 *     the integer whose bits are the keys.  The sign is that of the nonzero
 *     coefficient with the smallest exponent.
 *
 * The expansion below is the literal definition: it multiplies out
 * prod_c (M[pi(c)][c] + eps-term) for every permutation pi and every subset
 * of columns taking the eps-term, and accumulates coefficients per exponent.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

static int perm_parity(const int *p, int n) {
    int inv = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (p[i] > p[j]) ++inv;
    return (inv & 1) ? -1 : 1;
}

/* next permutation in lexicographic order; returns 0 after the last one */
static int next_perm(int *p, int n) {
    int i = n - 2;
    while (i >= 0 && p[i] >= p[i + 1]) --i;
    if (i < 0) return 0;
    int j = n - 1;
    while (p[j] <= p[i]) --j;
    int t = p[i]; p[i] = p[j]; p[j] = t;
    for (int a = i + 1, b = n - 1; a < b; ++a, --b) { t = p[a]; p[a] = p[b]; p[b] = t; }
    return 1;
}

/*
 * SoS sign of det(M + E(eps)), M an n x n integer matrix stored column-major
 * (M[c*n + r] = component r of the c-th column), columns already sorted by
 * increasing vertex id.  n <= 3.  Returns +1 or -1 (never 0).
 *
 * oracle_sos_det_sign_expand is the literal definition (every coefficient of
 * the expansion); oracle_sos_det_sign returns the same sign, reading the
 * eps^0 coefficient first.
 */
int oracle_sos_det_sign_expand(int n, const int64_t *M) {
    if (n < 1 || n > 3) return 0;
    i128 coef[1 << 9];
    const int nmask = 1 << (n * n);
    memset(coef, 0, sizeof(i128) * (size_t)nmask);
    int p[3];
    for (int i = 0; i < n; ++i) p[i] = i;
    do {
        const int sgn = perm_parity(p, n);
        for (int C = 0; C < (1 << n); ++C) {
            i128 prod = sgn;
            int mask = 0;
            for (int c = 0; c < n; ++c) {
                const int r = p[c];
                if ((C >> c) & 1) mask |= 1 << (c * n + r);
                else prod *= (i128)M[c * n + r];
            }
            coef[mask] += prod;
        }
    } while (next_perm(p, n));
    for (int m = 0; m < nmask; ++m)
        if (coef[m] != 0) return coef[m] > 0 ? 1 : -1;
    return 0; /* unreachable: the all-perturbed terms have coefficient +-1 */
}

int oracle_sos_det_sign(int n, const int64_t *M) {
    if (n < 1 || n > 3) return 0;
    int p[3];
    /* The coefficient of eps^0 (no entry perturbed) is det(M) itself.  It is
       the coefficient of smallest exponent, so when it is nonzero its sign is
       the answer and the higher-order coefficients are never consulted. */
    i128 det0 = 0;
    for (int i = 0; i < n; ++i) p[i] = i;
    do {
        i128 prod = perm_parity(p, n);
        for (int c = 0; c < n; ++c) prod *= (i128)M[c * n + p[c]];
        det0 += prod;
    } while (next_perm(p, n));
    if (det0 != 0) return det0 > 0 ? 1 : -1;
    return oracle_sos_det_sign_expand(n, M);
}

/*
 * Puncture test of one face.  V[k*n + r] = component r of the vector at the
 * k-th vertex, vertices sorted by increasing global id.  Returns 1 if
 * punctured, 0 otherwise.
 */
int oracle_face_punctured(int n, const int64_t *V) {
    int64_t M[9];
    int ref = 0;
    for (int k = 0; k <= n; ++k) {
        int c = 0;
        for (int j = 0; j <= n; ++j) {
            if (j == k) continue;
            for (int r = 0; r < n; ++r) M[c * n + r] = V[j * n + r];
            ++c;
        }
        int s = oracle_sos_det_sign(n, M);
        int val = (k & 1) ? -s : s;
        if (k == 0) ref = val;
        else if (val != ref) return 0;
    }
    return 1;
}

/* row-major strides of the spacetime grid: stride[a] = prod_{b<a} dims[b] */
static void grid_strides(int n, const int64_t *dims, int64_t *stride) {
    stride[0] = 1;
    for (int a = 1; a <= n; ++a) stride[a] = stride[a - 1] * dims[a - 1];
}

/*
 * Test every face whose base vertex is g (all ntypes types; a type exists
 * iff its last vertex base + bits(chain[n-1]) lies in the grid).  Punctured
 * face ids g*ntypes + type go to out[0..] in type order while they fit in
 * cap; returns how many were punctured.
 */
static int scan_vertex(int n, const int64_t *dims, const int64_t *stride, const int64_t *G, int ntypes,
                       const int32_t *chains, int64_t g, int64_t *out, int64_t cap) {
    const int d = n + 1;
    int64_t V[12];
    int64_t c[4];
    int count = 0;
    for (int a = 0; a < d; ++a) c[a] = (g / stride[a]) % dims[a];
    for (int tt = 0; tt < ntypes; ++tt) {
        const int32_t *ch = chains + (size_t)tt * n;
        const int32_t last = ch[n - 1];
        int ok = 1;
        for (int a = 0; a < d; ++a)
            if (((last >> a) & 1) && c[a] + 1 >= dims[a]) ok = 0;
        if (!ok) continue;
        for (int k = 0; k <= n; ++k) {
            int64_t v = g;
            if (k > 0)
                for (int a = 0; a < d; ++a)
                    if ((ch[k - 1] >> a) & 1) v += stride[a];
            for (int r = 0; r < n; ++r) V[k * n + r] = G[v * n + r];
        }
        if (oracle_face_punctured(n, V)) {
            if (count < cap) out[count] = g * ntypes + tt;
            ++count;
        }
    }
    return count;
}

/*
 * Enumerate every face (n-simplex) of the Kuhn spacetime mesh whose base
 * vertex lies in time slices [t_lo, t_hi) and test it.
 *
 *   dims[0..n-1] : spatial extents (x, y[, z]); dims[n] = nt
 *   G            : int64 vectors, G[g*n + r], g = row-major spacetime vertex id
 *   chains       : ntypes x n bitmasks (axis bit a; bit n is time); face type
 *                  tt has vertices base + bits(chains[tt*n + i]), i = -1..n-1
 *   out          : receives punctured face ids g*ntypes + type, ascending
 *
 * Returns the number of punctured faces (entries beyond cap are not written).
 */
int64_t oracle_scan(int n, const int64_t *dims, const int64_t *G, int ntypes,
                    const int32_t *chains, int64_t t_lo, int64_t t_hi,
                    int64_t *out, int64_t cap) {
    int64_t stride[4];
    grid_strides(n, dims, stride);
    const int64_t slice = stride[n];
    int64_t count = 0;
    int64_t buf[64];
    for (int64_t g = t_lo * slice; g < t_hi * slice; ++g) {
        const int k = scan_vertex(n, dims, stride, G, ntypes, chains, g, buf, 64);
        for (int i = 0; i < k; ++i, ++count)
            if (count < cap) out[count] = buf[i];
    }
    return count;
}

/*
 * The same enumeration over `threads` OpenMP threads (when the library is
 * built with OpenMP; otherwise one thread).  The base vertices are cut into
 * contiguous chunks; each chunk collects its punctured ids in vertex order
 * into a buffer of its own, and the buffers are concatenated in chunk order,
 * so the output is identical to oracle_scan's.
 */
int64_t oracle_scan_mt(int n, const int64_t *dims, const int64_t *G, int ntypes,
                       const int32_t *chains, int64_t t_lo, int64_t t_hi,
                       int64_t *out, int64_t cap, int threads) {
    int64_t stride[4];
    grid_strides(n, dims, stride);
    const int64_t slice = stride[n];
    const int64_t g0 = t_lo * slice, g1 = t_hi * slice;
    if (threads < 1) threads = 1;
    const int64_t nchunk = (int64_t)threads * 16;
    const int64_t span = (g1 - g0 + nchunk - 1) / nchunk;
    int64_t **bufs = (int64_t **)calloc((size_t)nchunk, sizeof(int64_t *));
    int64_t *cnt = (int64_t *)calloc((size_t)nchunk, sizeof(int64_t));
    int failed = 0;
    if (!bufs || !cnt) { free(bufs); free(cnt); return -1; }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
    for (int64_t ch = 0; ch < nchunk; ++ch) {
        const int64_t a = g0 + ch * span, b = a + span < g1 ? a + span : g1;
        int64_t bcap = 1024, k = 0;
        int64_t *bp = (int64_t *)malloc((size_t)bcap * sizeof(int64_t));
        int64_t tmp[64];
        for (int64_t g = a; g < b && bp; ++g) {
            const int m = scan_vertex(n, dims, stride, G, ntypes, chains, g, tmp, 64);
            if (k + m > bcap) {
                bcap = 2 * (k + m);
                int64_t *nb = (int64_t *)realloc(bp, (size_t)bcap * sizeof(int64_t));
                if (!nb) { free(bp); bp = NULL; break; }
                bp = nb;
            }
            for (int i = 0; i < m; ++i) bp[k++] = tmp[i];
        }
        if (!bp) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
        bufs[ch] = bp;
        cnt[ch] = k;
    }
    int64_t count = 0;
    for (int64_t ch = 0; ch < nchunk; ++ch) {
        for (int64_t i = 0; i < cnt[ch] && bufs[ch]; ++i, ++count)
            if (count < cap) out[count] = bufs[ch][i];
        free(bufs[ch]);
    }
    free(bufs);
    free(cnt);
    return failed ? -1 : count;
}

/* threads available to the OpenMP scan (1 when built without OpenMP) */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Test a list of faces given by id (for sampled checks at full size).
 * res[i] = 1 if face_ids[i] is punctured, 0 if not, -1 if it does not exist.
 */
void oracle_test_faces(int n, const int64_t *dims, const int64_t *G, int ntypes,
                       const int32_t *chains, const int64_t *face_ids, int64_t count,
                       int8_t *res) {
    const int d = n + 1;
    int64_t stride[4];
    stride[0] = 1;
    for (int a = 1; a < d; ++a) stride[a] = stride[a - 1] * dims[a - 1];
    int64_t V[12];
    int64_t c[4];
    for (int64_t i = 0; i < count; ++i) {
        const int64_t g = face_ids[i] / ntypes;
        const int tt = (int)(face_ids[i] % ntypes);
        for (int a = 0; a < d; ++a) c[a] = (g / stride[a]) % dims[a];
        const int32_t *ch = chains + (size_t)tt * n;
        int ok = 1;
        for (int a = 0; a < d; ++a)
            if (((ch[n - 1] >> a) & 1) && c[a] + 1 >= dims[a]) ok = 0;
        if (!ok) { res[i] = -1; continue; }
        for (int k = 0; k <= n; ++k) {
            int64_t v = g;
            if (k > 0)
                for (int a = 0; a < d; ++a)
                    if ((ch[k - 1] >> a) & 1) v += stride[a];
            for (int r = 0; r < n; ++r) V[k * n + r] = G[v * n + r];
        }
        res[i] = (int8_t)oracle_face_punctured(n, V);
    }
}
