// Isovolume tracking on the simplicial spacetime mesh (paper Sec. 6.1;
// Algorithm 1, right column), 2D + time and 3D + time.
//
//   k_iso_bits   dense, HBM-bound: one pass over the field; bit x of word k
//                of row (t, z, y) = [f >= c] for x = 32 k + bit (a sample
//                equal to c counts as above: its symbolic perturbation is a
//                positive infinitesimal).  Non-finite samples are flagged.
//   k_iso_emit   per (row, word) item: the intersected edges of its 32 base
//                vertices, one bit word per edge mask m (vertex bits XOR
//                the bits of the vertex one step along m); an ordered
//                single-pass scan (decoupled look-back) gives every item its
//                first edge and first "owner" (a vertex with an intersected
//                edge of its own); the edges are written in id order with
//                their crossing points, and every owner's first edge index
//                and edge mask.
//   k_iso_link   per owner whose unit cube lies in the grid: the cube's
//                cells (pentachora / tetrahedra, one per ordering of the
//                axes) unite their intersected edges -- first in a small
//                union-find over the cube's 3^d - 2^d edge slots, then one
//                global union (lock-free) per edge of each local piece.
//   k_iso_label  label = smallest edge id of the piece; host-layout records.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "../../include/ftk.h"
#include "ftk_internal.h"
#include "ftk_tma.cuh"

struct ftk_iso_result {
    ftk_iso_point *data;
    size_t count;
};

namespace ftk {
namespace {

constexpr int INT = 256;                   // threads per block
constexpr uint32_t ALL = 0xffffffffu;
constexpr int ISO_UF_LIMIT = 1 << 22;      // bound of the union-find loops

enum : unsigned {
    IST_RANGE = 1u,      // a non-finite sample
    IST_OVERFLOW = 2u,   // edge or owner capacity exceeded (counts still exact)
    IST_TIMEOUT = 4u,    // a bounded device loop gave up
    IST_BIG = 8u,        // more than 2^31 - 1 intersected edges
};

struct IsoGrid {
    const float *f;      // f[t][z][y][x], rows of nx floats
    int nx, ny, nz, nt;  // nz = 1 in 2D
    int W;               // bit words per row: ceil(nx / 32)
    long long rows;      // nt * nz * ny
    float c_up;          // smallest float >= isovalue: f >= c  <=>  f >= c_up
    float c_hi, c_lo;    // isovalue ~= c_hi + c_lo
};

struct IsoCtr {
    unsigned status;
    unsigned pad;
    long long edges;               // intersected edges (set by the last tile)
    long long owners;              // vertices owning an intersected edge
    unsigned long long tiles;      // tiles handed out by the emit kernel
    unsigned long long edges_chk;  // 64-bit running total of the edges (range check)
};

struct IsoWork {
    IsoCtr *ctr;
    uint32_t *bits;                // [items] above bits
    uint32_t *obits;               // [items] owners among the item's vertices
    int *item_own;                 // [items] owners before the item
    unsigned long long *tile;      // [ntiles] look-back states
    long long *own_g;              // [ocap] vertex id of each owner
    int *own_first;                // [ocap] its first edge index
    uint16_t *own_mask;            // [ocap] its intersected edge masks (bit m - 1)
    long long *id;                 // [cap] edge ids, sorted
    float4 *off;                   // [cap] crossing point - base vertex (x, y, z, t)
    int *parent;                   // [cap] union-find
    ftk_iso_point *rec;            // [cap] host-layout records
    long long cap, ocap;
};

// Compile-time tables of a unit d-cube: its Kuhn edges (corner pairs a < b
// with a a subset of b; a slot per pair) and its cells (one chain of corners
// per ordering of the d axes).
template <int N>
struct IsoTables {
    static constexpr int D = N + 1, NC = 1 << D;
    static constexpr int NS = N == 2 ? 19 : 65;      // 3^d - 2^d
    static constexpr int NCELL = N == 2 ? 6 : 24;    // d!
    uint8_t slot[NC][NC];
    uint8_t sa[NS], sb[NS];
    uint8_t chain[NCELL][D + 1];
    __host__ __device__ constexpr IsoTables() : slot{}, sa{}, sb{}, chain{} {
        int s = 0;
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) slot[a][b] = 255;
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b)
                if (a != b && (a & b) == a) {
                    slot[a][b] = (uint8_t)s;
                    sa[s] = (uint8_t)a;
                    sb[s] = (uint8_t)b;
                    ++s;
                }
        int tuples = 1;
        for (int i = 0; i < D; ++i) tuples *= D;
        int p = 0;
        for (int code = 0; code < tuples; ++code) {
            int dig[D] = {};
            int c = code, used = 0;
            bool ok = true;
            for (int j = D - 1; j >= 0; --j) {
                dig[j] = c % D;
                c /= D;
                if ((used >> dig[j]) & 1) ok = false;
                used |= 1 << dig[j];
            }
            if (!ok) continue;
            chain[p][0] = 0;
            for (int k = 0; k < D; ++k) chain[p][k + 1] = (uint8_t)(chain[p][k] | (1 << dig[k]));
            ++p;
        }
    }
};

__constant__ IsoTables<2> c_iso2 = IsoTables<2>();
__constant__ IsoTables<3> c_iso3 = IsoTables<3>();
template <int N> __device__ __forceinline__ const IsoTables<N> &iso_tables();
template <> __device__ __forceinline__ const IsoTables<2> &iso_tables<2>() { return c_iso2; }
template <> __device__ __forceinline__ const IsoTables<3> &iso_tables<3>() { return c_iso3; }

// element offset of the step along edge mask m from a vertex (bit N = t)
template <int N>
__device__ __forceinline__ long long iso_step(const IsoGrid &G, int m) {
    const long long sy = G.nx, sz = (long long)G.ny * G.nx, st = (long long)G.nz * G.ny * G.nx;
    return (m & 1) + ((m >> 1) & 1) * sy + (N == 3 ? ((m >> 2) & 1) * sz : 0) + ((m >> N) & 1) * st;
}
// row offset of the step along the y / z / t bits of m
template <int N>
__device__ __forceinline__ long long iso_row_step(const IsoGrid &G, int m) {
    return ((m >> 1) & 1) + (N == 3 ? ((m >> 2) & 1) * (long long)G.ny : 0) +
           ((m >> N) & 1) * (long long)G.nz * G.ny;
}

// w = f - c for c = c_hi + c_lo: the exact difference f - c_hi as a float
// pair (two-sum, Knuth), then the low parts
__device__ __forceinline__ float iso_w(float v, float c_hi, float c_lo) {
    const float s = __fadd_rn(v, -c_hi);
    const float bb = __fadd_rn(s, -v);
    const float e = __fadd_rn(__fadd_rn(v, -__fadd_rn(s, -bb)), __fadd_rn(-c_hi, -bb));
    return __fadd_rn(s, __fadd_rn(e, -c_lo));
}

// ---------------------------------------------------------------------------
// k_iso_bits: one warp per group of 8 consecutive (row, word) items; all
// loads of a group are issued before its ballots
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(INT) k_iso_bits(IsoGrid G, IsoWork W) {
    constexpr int U = 8;
    const long long items = G.rows * G.W;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * INT) >> 5;
    bool bad = false;
    for (long long it0 = (((long long)blockIdx.x * INT + threadIdx.x) >> 5) * U; it0 < items; it0 += nwarps * U) {
        long long row = it0 / G.W;
        int k = (int)(it0 - row * G.W);
        float v[U];
        bool in[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int x = k * 32 + lane;
            in[u] = it0 + u < items && x < G.nx;
            v[u] = in[u] ? __ldg(G.f + row * G.nx + x) : 0.0f;
            if (++k == G.W) {
                k = 0;
                ++row;
            }
        }
        uint32_t mine = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            bad |= in[u] && !(fabsf(v[u]) <= FLT_MAX);
            const uint32_t w = __ballot_sync(ALL, in[u] && v[u] >= G.c_up);
            if (lane == u) mine = w;
        }
        if (lane < U && it0 + lane < items) W.bits[it0 + lane] = mine;
    }
    if (__any_sync(ALL, bad) && lane == 0) atomicOr(&W.ctr->status, IST_RANGE);
}

// edge words of item (row, k): X[m-1] bit b = vertex x = 32 k + b owns an
// intersected edge along m (m = 1 .. 2^d - 1)
template <int N>
__device__ __forceinline__ void iso_item_words(const IsoGrid &G, const uint32_t *bits, long long row, int k,
                                               uint32_t (&X)[(1 << (N + 1)) - 1]) {
    constexpr int D = N + 1, E = (1 << D) - 1;
    const long long ny = G.ny, nz = G.nz;
    const long long t = row / (ny * nz);
    const long long rz = row - t * ny * nz;
    const int z = (int)(rz / ny), y = (int)(rz - (long long)z * ny);
    const int x0 = 32 * k;
    // columns that can step +x, and columns inside the grid
    const int lx = G.nx - 1 - x0, lin = G.nx - x0;
    const uint32_t vx = lx >= 32 ? ALL : lx <= 0 ? 0u : (1u << lx) - 1u;
    const uint32_t vin = lin >= 32 ? ALL : (1u << lin) - 1u;
    const uint32_t A = bits[row * G.W + k];
#pragma unroll
    for (int m = 1; m <= E; ++m) {
        const bool ok = (!((m >> 1) & 1) || y + 1 < G.ny) && (N != 3 || !((m >> 2) & 1) || z + 1 < G.nz) &&
                        (!((m >> N) & 1) || t + 1 < G.nt);
        if (!ok) {
            X[m - 1] = 0u;
            continue;
        }
        const long long r2 = row + iso_row_step<N>(G, m);
        uint32_t B = bits[r2 * G.W + k];
        if (m & 1) {
            const uint32_t nxt = k + 1 < G.W ? bits[r2 * G.W + k + 1] : 0u;
            B = (B >> 1) | (nxt << 31);
            X[m - 1] = (A ^ B) & vx;
        } else {
            X[m - 1] = (A ^ B) & vin;
        }
    }
}

// block-wide exclusive scan of unsigned 64-bit values
__device__ __forceinline__ unsigned long long iso_block_scan(unsigned long long v, unsigned long long *red,
                                                             unsigned long long &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(ALL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < INT / 32 ? red[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < INT / 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(ALL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < INT / 32) red[lane] = w;
    }
    __syncthreads();
    const unsigned long long before = warp ? red[warp - 1] : 0ull;
    total = red[INT / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// Decoupled look-back across tiles (Merrill & Garland 2016): the state word
// of a tile holds its total (flag 1) or inclusive prefix (flag 2) in bits
// 0-61.  Called by one full warp; returns the exclusive prefix of tile t.
constexpr unsigned long long LB_AGG = 1ull << 62, LB_INC = 2ull << 62, LB_VAL = (1ull << 62) - 1;
__device__ unsigned long long iso_lookback(unsigned long long *tile_state, long long t, unsigned long long total,
                                           unsigned *status) {
    volatile unsigned long long *st = tile_state;
    const int lane = threadIdx.x & 31;
    if (lane == 0) st[t] = (t == 0 ? LB_INC : LB_AGG) | total;
    if (t == 0) return 0;
    unsigned long long ex = 0;
    long long hi = t - 1;
    const long long t0 = clock64();
    while (true) {
        const long long j = hi - lane;
        unsigned long long v = LB_INC;
        if (j >= 0) v = st[j];
        if (__any_sync(ALL, (v >> 62) == 0)) {
            if (clock64() - t0 > WAIT_CYCLES) {
                if (lane == 0) atomicOr(status, IST_TIMEOUT);
                break;
            }
            __nanosleep(32);
            continue;
        }
        const unsigned inc = __ballot_sync(ALL, (v >> 62) == 2);
        const int stop = inc ? __ffs(inc) - 1 : 31;
        unsigned long long x = lane <= stop ? (v & LB_VAL) : 0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(ALL, x, o);
        ex += x;
        if (inc) break;
        hi -= 32;
    }
    if (lane == 0) st[t] = LB_INC | ((ex + total) & LB_VAL);
    return ex;
}

// ---------------------------------------------------------------------------
// k_iso_emit: blocks claim tiles of INT consecutive items in order.  Counts
// travel packed: edges in bits 0-30, owners in bits 31-61 (each total stays
// below 2^31, checked through a separate 64-bit sum).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(INT) k_iso_emit(IsoGrid G, IsoWork W) {
    constexpr int D = N + 1, E = (1 << D) - 1;
    __shared__ unsigned long long red[INT / 32 + 1];
    __shared__ unsigned long long sh[2];
    const long long items = G.rows * G.W;
    const long long ntiles = (items + INT - 1) / INT;
    unsigned *status = &W.ctr->status;
    while (true) {
        if (threadIdx.x == 0) sh[1] = atomicAdd(&W.ctr->tiles, 1ull);
        __syncthreads();
        const long long t = (long long)sh[1];
        if (t >= ntiles) break;
        const long long it = t * INT + threadIdx.x;
        const bool have = it < items;
        uint32_t X[E];
        long long row = 0;
        int k = 0;
        if (have) {
            row = it / G.W;
            k = (int)(it - row * G.W);
            iso_item_words<N>(G, W.bits, row, k, X);
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) X[m] = 0u;
        }
        uint32_t own = 0;
        int ne = 0;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            own |= X[m];
            ne += __popc(X[m]);
        }
        const int no = __popc(own);
        unsigned long long tot;
        const unsigned long long ex = iso_block_scan((unsigned long long)ne | ((unsigned long long)no << 31), red, tot);
        if (threadIdx.x < 32) {
            const unsigned long long before = iso_lookback(W.tile, t, tot, status);
            if (threadIdx.x == 0) {
                sh[0] = before;
                if ((tot & 0x7fffffffull) != 0) atomicAdd(&W.ctr->edges_chk, tot & 0x7fffffffull);
                if (t == ntiles - 1) {
                    W.ctr->edges = (long long)((before + tot) & 0x7fffffffull);
                    W.ctr->owners = (long long)((before + tot) >> 31);
                }
            }
        }
        __syncthreads();
        const unsigned long long pre = sh[0] + ex;
        long long e0 = (long long)(pre & 0x7fffffffull);
        long long o0 = (long long)(pre >> 31);
        if (have) {
            W.obits[it] = own;
            W.item_own[it] = (int)o0;
        }
        if (have && own) {
            const bool fits = e0 + ne <= W.cap && o0 + no <= W.ocap;
            if (!fits) atomicOr(status, IST_OVERFLOW);
            const long long g0 = row * G.nx + 32 * k;
            uint32_t rest = own;
            while (fits && rest) {
                const int b = __ffs(rest) - 1;
                rest &= rest - 1;
                const long long g = g0 + b;
                const float w0 = iso_w(__ldg(G.f + g), G.c_hi, G.c_lo);
                uint32_t mask = 0;
                const long long first = e0;
#pragma unroll
                for (int m = 1; m <= E; ++m) {
                    if (!((X[m - 1] >> b) & 1u)) continue;
                    mask |= 1u << (m - 1);
                    const float w1 = iso_w(__ldg(G.f + g + iso_step<N>(G, m)), G.c_hi, G.c_lo);
                    const float den = w0 - w1;
                    float mu = den != 0.0f ? w0 / den : 0.0f;
                    mu = fminf(fmaxf(mu, 0.0f), 1.0f);
                    W.id[e0] = g * E + (m - 1);
                    W.off[e0] = make_float4((m & 1) ? mu : 0.0f, ((m >> 1) & 1) ? mu : 0.0f,
                                            N == 3 && ((m >> 2) & 1) ? mu : 0.0f, ((m >> N) & 1) ? mu : 0.0f);
                    W.parent[e0] = (int)e0;
                    ++e0;
                }
                W.own_g[o0] = g;
                W.own_first[o0] = (int)first;
                W.own_mask[o0] = (uint16_t)mask;
                ++o0;
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int iso_find(int *parent, int x, unsigned *status) {
    for (int it = 0; it < ISO_UF_LIMIT; ++it) {
        const int p = *(volatile int *)&parent[x];
        if (p == x) return x;
        const int gp = *(volatile int *)&parent[p];
        if (gp != p) *(volatile int *)&parent[x] = gp;   // path halving
        x = gp;
    }
    atomicOr(status, IST_TIMEOUT);
    return x;
}

__device__ __forceinline__ void iso_unite(int *parent, int a, int b, unsigned *status) {
    for (int it = 0; it < ISO_UF_LIMIT; ++it) {
        a = iso_find(parent, a, status);
        b = iso_find(parent, b, status);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        // the larger root under the smaller: roots stay component minima
        const int old = atomicCAS(&parent[a], a, b);
        if (old == a) return;
        a = old;
    }
    atomicOr(status, IST_TIMEOUT);
}

// ---------------------------------------------------------------------------
// k_iso_link: one thread per owner whose unit cube lies in the grid
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(INT) k_iso_link(IsoGrid G, IsoWork W) {
    using Tb = IsoTables<N>;
    constexpr int D = N + 1, NC = 1 << D, NS = Tb::NS, NCELL = Tb::NCELL;
    __shared__ uint8_t s_slot[NC][NC];
    __shared__ uint8_t s_sa[NS], s_sb[NS];
    __shared__ uint8_t s_chain[NCELL][D + 1];
    __shared__ uint8_t lp[NS][INT];   // per-thread local union-find over the cube's edge slots
    for (int i = threadIdx.x; i < NC * NC; i += INT) s_slot[i / NC][i % NC] = iso_tables<N>().slot[i / NC][i % NC];
    for (int i = threadIdx.x; i < NS; i += INT) {
        s_sa[i] = iso_tables<N>().sa[i];
        s_sb[i] = iso_tables<N>().sb[i];
    }
    for (int i = threadIdx.x; i < NCELL * (D + 1); i += INT)
        s_chain[i / (D + 1)][i % (D + 1)] = iso_tables<N>().chain[i / (D + 1)][i % (D + 1)];
    __syncthreads();
    if (W.ctr->status & (IST_OVERFLOW | IST_RANGE | IST_BIG)) return;
    const long long no = W.ctr->owners;
    unsigned *status = &W.ctr->status;
    const int me = threadIdx.x;
    for (long long s = blockIdx.x * (long long)INT + threadIdx.x; s < no; s += (long long)gridDim.x * INT) {
        const long long g = W.own_g[s];
        const long long row = g / G.nx;
        const int x = (int)(g - row * G.nx);
        const long long t = row / ((long long)G.ny * G.nz);
        const long long rz = row - t * G.ny * G.nz;
        const int z = (int)(rz / G.ny), y = (int)(rz - (long long)z * G.ny);
        if (x + 1 >= G.nx || y + 1 >= G.ny || (N == 3 && z + 1 >= G.nz) || t + 1 >= G.nt) continue;
        // above bits of the cube's corners (corner index = axis mask)
        uint32_t cb = 0;
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const long long r2 = row + iso_row_step<N>(G, a);
            const int xa = x + (a & 1);
            cb |= ((W.bits[r2 * G.W + (xa >> 5)] >> (xa & 31)) & 1u) << a;
        }
        // local union-find over the intersected edge slots, through the cells
        uint64_t hit_lo = 0;   // slots 0-63
        uint32_t hit_hi = 0;   // slot 64 (3D)
#pragma unroll 1
        for (int p = 0; p < NCELL; ++p) {
            int c[D + 1];
            uint32_t cm = 0;
#pragma unroll
            for (int q = 0; q <= D; ++q) {
                c[q] = s_chain[p][q];
                cm |= 1u << c[q];
            }
            const uint32_t up = cb & cm;
            if (up == 0 || up == cm) continue;
            int first = -1;
#pragma unroll
            for (int i = 0; i <= D; ++i)
#pragma unroll
                for (int j = i + 1; j <= D; ++j) {
                    if (((cb >> c[i]) ^ (cb >> c[j])) & 1u) {
                        const int sl = s_slot[c[i]][c[j]];
                        const bool seen = sl < 64 ? (hit_lo >> sl) & 1ull : hit_hi & 1u;
                        if (!seen) {
                            lp[sl][me] = (uint8_t)sl;
                            if (sl < 64) hit_lo |= 1ull << sl;
                            else hit_hi |= 1u;
                        }
                        if (first < 0) {
                            first = sl;
                        } else {
                            // local union: the larger root under the smaller
                            int ra = first, rb = sl;
                            while (lp[ra][me] != ra) ra = lp[ra][me];
                            while (lp[rb][me] != rb) rb = lp[rb][me];
                            if (ra != rb) {
                                if (ra < rb) lp[rb][me] = (uint8_t)ra;
                                else lp[ra][me] = (uint8_t)rb;
                            }
                        }
                    }
                }
        }
        // one global union per edge of each local piece, with its local root;
        // edge indices through the owner lists of the edges' lower corners
        int cfirst[NC];
        uint32_t cmask[NC];
        uint32_t have = 0;
        auto gidx = [&](int sl) -> int {
            const int a = s_sa[sl], b = s_sb[sl];
            if (!((have >> a) & 1u)) {
                const long long r2 = row + iso_row_step<N>(G, a);
                const int xa = x + (a & 1);
                const long long item = r2 * G.W + (xa >> 5);
                const int bit = xa & 31;
                const long long o = W.item_own[item] + __popc(W.obits[item] & ((1u << bit) - 1u));
                cfirst[a] = W.own_first[o];
                cmask[a] = W.own_mask[o];
                have |= 1u << a;
            }
            const int m = a ^ b;
            return cfirst[a] + __popc(cmask[a] & ((1u << (m - 1)) - 1u));
        };
        for (int sl = 0; sl < NS; ++sl) {
            const bool hit = sl < 64 ? (hit_lo >> sl) & 1ull : hit_hi & 1u;
            if (!hit) continue;
            int r = sl;
            while (lp[r][me] != r) r = lp[r][me];
            if (r != sl) iso_unite(W.parent, gidx(sl), gidx(r), status);
        }
    }
}

// ---------------------------------------------------------------------------
// k_iso_label: label = id of the component's root (its smallest index, so
// its smallest id); host-layout records
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(INT) k_iso_label(IsoGrid G, IsoWork W) {
    constexpr int D = N + 1, E = (1 << D) - 1;
    if (W.ctr->status & (IST_OVERFLOW | IST_RANGE | IST_BIG)) return;
    const long long P = W.ctr->edges;
    unsigned *status = &W.ctr->status;
    for (long long i = blockIdx.x * (long long)INT + threadIdx.x; i < P; i += (long long)gridDim.x * INT) {
        const int r = iso_find(W.parent, (int)i, status);
        const long long id = W.id[i];
        const long long g = id / E;
        const int m = (int)(id - g * E) + 1;
        const long long row = g / G.nx;
        const int x = (int)(g - row * G.nx);
        const long long tt = row / ((long long)G.ny * G.nz);
        const long long rz = row - tt * G.ny * G.nz;
        const int z = (int)(rz / G.ny), y = (int)(rz - (long long)z * G.ny);
        ftk_iso_point p;
        p.edge_id = id;
        p.label = W.id[r];
        p.base[0] = x;
        p.base[1] = y;
        p.base[2] = z;
        p.base[3] = (int)tt;
        const float4 o = W.off[i];
        p.off[0] = o.x;
        p.off[1] = o.y;
        p.off[2] = o.z;
        p.off[3] = o.w;
        p.ordinal = ((m >> N) & 1) ? 0 : 1;
        p.ndim = (uint8_t)N;
        for (int q = 0; q < 6; ++q) p.reserved[q] = 0;
        W.rec[i] = p;
    }
}

int num_sms() {
    static const int n = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return sms > 0 ? sms : 148;
    }();
    return n;
}

}  // namespace
}  // namespace ftk

using namespace ftk;

struct ftk_iso_plan {
    int ndim;
    int device;
    IsoGrid G;
    IsoWork W;
    IsoCtr *h_ctr;          // pinned mirror of the counters
    float *d_input;         // copy of a host field
    cudaStream_t stream;
    cudaEvent_t copy_ev;
    const float *last_dev;  // the device field the last run read
    double isovalue;
    long long items, ntiles, nverts;
    bool executed;
    cudaEvent_t ev[5];      // bounds of the four kernels of the last run
};

namespace {

#define ISO_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e__ = (call);                           \
        if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
    } while (0)

void iso_free_caps(IsoWork &W) {
    cudaFree(W.own_g);
    cudaFree(W.own_first);
    cudaFree(W.own_mask);
    cudaFree(W.id);
    cudaFree(W.off);
    cudaFree(W.parent);
    cudaFree(W.rec);
    W.own_g = nullptr;
    W.own_first = nullptr;
    W.own_mask = nullptr;
    W.id = nullptr;
    W.off = nullptr;
    W.parent = nullptr;
    W.rec = nullptr;
}

ftk_status iso_alloc_caps(IsoWork &W, long long cap, long long ocap) {
    iso_free_caps(W);
    W.cap = W.ocap = 0;
    cap = std::min<long long>(std::max<long long>(cap, 1024), INT32_MAX);
    ocap = std::min<long long>(std::max<long long>(ocap, 1024), INT32_MAX);
    if (cudaMalloc(&W.own_g, sizeof(long long) * ocap) != cudaSuccess ||
        cudaMalloc(&W.own_first, sizeof(int) * ocap) != cudaSuccess ||
        cudaMalloc(&W.own_mask, sizeof(uint16_t) * ocap) != cudaSuccess ||
        cudaMalloc(&W.id, sizeof(long long) * cap) != cudaSuccess ||
        cudaMalloc(&W.off, sizeof(float4) * cap) != cudaSuccess ||
        cudaMalloc(&W.parent, sizeof(int) * cap) != cudaSuccess ||
        cudaMalloc(&W.rec, sizeof(ftk_iso_point) * cap) != cudaSuccess) {
        cudaGetLastError();
        iso_free_caps(W);
        return fail(FTK_ERR_NOMEM, "device allocation of the isovolume capacity failed");
    }
    W.cap = cap;
    W.ocap = ocap;
    return FTK_OK;
}

void iso_destroy(ftk_iso_plan *pl) {
    if (!pl) return;
    iso_free_caps(pl->W);
    cudaFree(pl->W.ctr);
    cudaFree(pl->W.bits);
    cudaFree(pl->W.obits);
    cudaFree(pl->W.item_own);
    cudaFree(pl->W.tile);
    cudaFree(pl->d_input);
    if (pl->h_ctr) cudaFreeHost(pl->h_ctr);
    if (pl->copy_ev) cudaEventDestroy(pl->copy_ev);
    for (cudaEvent_t e : pl->ev)
        if (e) cudaEventDestroy(e);
    delete pl;
}

// the isovalue as comparison threshold and float pair
ftk_status iso_set_value(IsoGrid &G, double c) {
    if (std::isnan(c)) return fail(FTK_ERR_ARG, "the isovalue is NaN");
    float up = (float)c;
    if ((double)up < c) up = std::nextafter(up, INFINITY);
    G.c_up = up;
    if (std::isfinite(c) && std::fabs(c) <= (double)FLT_MAX) {
        G.c_hi = (float)c;
        G.c_lo = (float)(c - (double)G.c_hi);
    } else {
        G.c_hi = (float)c;
        G.c_lo = 0.0f;
    }
    return FTK_OK;
}

ftk_status iso_launch(ftk_iso_plan *pl, const float *dev_f, cudaStream_t s) {
    pl->G.f = dev_f;
    IsoWork &W = pl->W;
    ISO_CUDA(cudaMemsetAsync(W.ctr, 0, sizeof(IsoCtr), s));
    ISO_CUDA(cudaMemsetAsync(W.tile, 0, sizeof(unsigned long long) * (size_t)pl->ntiles, s));
    const int sms = num_sms();
    const long long items = pl->items;
    const unsigned gb = (unsigned)std::max<long long>(1, std::min<long long>((items + 63) / 64, (long long)sms * 8));
    ISO_CUDA(cudaEventRecord(pl->ev[0], s));
    k_iso_bits<<<gb, INT, 0, s>>>(pl->G, W);
    ISO_CUDA(cudaEventRecord(pl->ev[1], s));
    const unsigned ge = (unsigned)std::max<long long>(1, std::min<long long>(pl->ntiles, (long long)sms * 4));
    const unsigned gl = (unsigned)std::max<long long>(1, std::min<long long>((W.ocap + INT - 1) / INT, (long long)sms * 8));
    const unsigned gL = (unsigned)std::max<long long>(1, std::min<long long>((W.cap + INT - 1) / INT, (long long)sms * 8));
    if (pl->ndim == 2) {
        k_iso_emit<2><<<ge, INT, 0, s>>>(pl->G, W);
        ISO_CUDA(cudaEventRecord(pl->ev[2], s));
        k_iso_link<2><<<gl, INT, 0, s>>>(pl->G, W);
        ISO_CUDA(cudaEventRecord(pl->ev[3], s));
        k_iso_label<2><<<gL, INT, 0, s>>>(pl->G, W);
    } else {
        k_iso_emit<3><<<ge, INT, 0, s>>>(pl->G, W);
        ISO_CUDA(cudaEventRecord(pl->ev[2], s));
        k_iso_link<3><<<gl, INT, 0, s>>>(pl->G, W);
        ISO_CUDA(cudaEventRecord(pl->ev[3], s));
        k_iso_label<3><<<gL, INT, 0, s>>>(pl->G, W);
    }
    ISO_CUDA(cudaEventRecord(pl->ev[4], s));
    ISO_CUDA(cudaGetLastError());
    pl->stream = s;
    pl->last_dev = dev_f;
    pl->executed = true;
    return FTK_OK;
}

// wait for the run, grow and re-run on overflow, check the status
ftk_status iso_settle(ftk_iso_plan *pl) {
    if (!pl->executed) return fail(FTK_ERR_STATE, "plan has not been executed");
    for (int attempt = 0; attempt < 6; ++attempt) {
        ISO_CUDA(cudaStreamSynchronize(pl->stream));
        ISO_CUDA(cudaMemcpy(pl->h_ctr, pl->W.ctr, sizeof(IsoCtr), cudaMemcpyDeviceToHost));
        const IsoCtr &c = *pl->h_ctr;
        if (c.status & IST_RANGE) return fail(FTK_ERR_RANGE, "a sample is non-finite");
        if (c.edges_chk > (unsigned long long)INT32_MAX)
            return fail(FTK_ERR_RANGE, "more than 2^31 - 1 intersected edges");
        if (c.status & IST_TIMEOUT) return fail(FTK_ERR_TIMEOUT, "a bounded device loop gave up");
        if (!(c.status & IST_OVERFLOW)) return FTK_OK;
        const long long need = c.edges, oneed = c.owners;
        ftk_status s = iso_alloc_caps(pl->W, std::max<long long>(need + need / 4 + 1024, pl->W.cap),
                                      std::max<long long>(oneed + oneed / 4 + 1024, pl->W.ocap));
        if (s != FTK_OK) return s;
        if ((s = iso_launch(pl, pl->last_dev, pl->stream)) != FTK_OK) return s;
    }
    return fail(FTK_ERR_NOMEM, "the isovolume capacity did not converge");
}

ftk_status iso_create(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t nt, ftk_iso_plan **out) {
    if (!out) return fail(FTK_ERR_ARG, "plan must be non-NULL");
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return fail(FTK_ERR_ARG, "ndim must be 2 or 3");
    if (ndim == 2) nz = 1;
    if (nx < 2 || ny < 2 || nt < 1 || (ndim == 3 && nz < 2))
        return fail(FTK_ERR_ARG, "every spatial extent must be >= 2 and nt >= 1");
    if (nx > INT32_MAX || ny > INT32_MAX || nz > INT32_MAX || nt > INT32_MAX)
        return fail(FTK_ERR_ARG, "extent too large");
    const double nv = (double)nx * ny * nz * nt;
    if (nv > 4e18 / 16) return fail(FTK_ERR_ARG, "grid too large");
    ftk_iso_plan *pl = new (std::nothrow) ftk_iso_plan();
    if (!pl) return fail(FTK_ERR_NOMEM, "host allocation failed");
    pl->ndim = ndim;
    cudaGetDevice(&pl->device);
    IsoGrid &G = pl->G;
    G.nx = (int)nx;
    G.ny = (int)ny;
    G.nz = (int)nz;
    G.nt = (int)nt;
    G.W = (int)((nx + 31) / 32);
    G.rows = (long long)nt * nz * ny;
    pl->nverts = G.rows * nx;
    pl->items = G.rows * G.W;
    pl->ntiles = (pl->items + INT - 1) / INT;
    IsoWork &W = pl->W;
    auto bad = [&](const char *what) {
        cudaGetLastError();
        iso_destroy(pl);
        return fail(FTK_ERR_NOMEM, what);
    };
    if (cudaMalloc(&W.ctr, sizeof(IsoCtr)) != cudaSuccess ||
        cudaMalloc(&W.bits, sizeof(uint32_t) * pl->items) != cudaSuccess ||
        cudaMalloc(&W.obits, sizeof(uint32_t) * pl->items) != cudaSuccess ||
        cudaMalloc(&W.item_own, sizeof(int) * pl->items) != cudaSuccess ||
        cudaMalloc(&W.tile, sizeof(unsigned long long) * pl->ntiles) != cudaSuccess)
        return bad("device allocation of the isovolume workspace failed");
    if (cudaHostAlloc(&pl->h_ctr, sizeof(IsoCtr), cudaHostAllocDefault) != cudaSuccess)
        return bad("pinned host allocation failed");
    if (cudaEventCreateWithFlags(&pl->copy_ev, cudaEventDisableTiming) != cudaSuccess)
        return bad("event creation failed");
    for (cudaEvent_t &e : pl->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bad("event creation failed");
    const long long cap0 = std::max<long long>(65536, pl->nverts / 16);
    const long long ocap0 = std::max<long long>(65536, pl->nverts / 64);
    if (iso_alloc_caps(W, cap0, ocap0) != FTK_OK) return bad("device allocation of the isovolume capacity failed");
    *out = pl;
    return FTK_OK;
}

ftk_status iso_execute(ftk_iso_plan *pl, const float *f, double c, cudaStream_t s) {
    if (!pl || !f) return fail(FTK_ERR_ARG, "plan and field must be non-NULL");
    ftk_status st = iso_set_value(pl->G, c);
    if (st != FTK_OK) return st;
    pl->isovalue = c;
    const float *src = f;
    if (!is_device_pointer(f)) {
        if (!pl->d_input && cudaMalloc(&pl->d_input, sizeof(float) * pl->nverts) != cudaSuccess) {
            cudaGetLastError();
            pl->d_input = nullptr;
            return fail(FTK_ERR_NOMEM, "device allocation of the input copy failed");
        }
        ISO_CUDA(cudaMemcpyAsync(pl->d_input, f, sizeof(float) * pl->nverts, cudaMemcpyHostToDevice, s));
        // the caller may reuse its buffer once this returns
        ISO_CUDA(cudaEventRecord(pl->copy_ev, s));
        ISO_CUDA(cudaEventSynchronize(pl->copy_ev));
        src = pl->d_input;
    }
    return iso_launch(pl, src, s);
}

ftk_status iso_download(ftk_iso_plan *pl, ftk_iso_result **out) {
    const long long P = pl->h_ctr->edges;
    ftk_iso_result *r = new (std::nothrow) ftk_iso_result;
    if (!r) return fail(FTK_ERR_NOMEM, "host allocation failed");
    r->count = (size_t)P;
    r->data = (ftk_iso_point *)std::malloc(std::max<size_t>(1, (size_t)P) * sizeof(ftk_iso_point));
    if (!r->data) {
        delete r;
        return fail(FTK_ERR_NOMEM, "host allocation failed");
    }
    if (P > 0) {
        cudaError_t e = cudaMemcpy(r->data, pl->W.rec, (size_t)P * sizeof(ftk_iso_point), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            std::free(r->data);
            delete r;
            return cuda_fail(e, "isovolume result download");
        }
    }
    *out = r;
    return FTK_OK;
}

}  // namespace

extern "C" {

ftk_status ftk_iso_plan_create(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t nt, ftk_iso_plan **plan) {
    return iso_create(ndim, nx, ny, nz, nt, plan);
}

ftk_status ftk_iso_plan_execute(ftk_iso_plan *plan, const float *f, double isovalue, void *cuda_stream) {
    return iso_execute(plan, f, isovalue, (cudaStream_t)cuda_stream);
}

ftk_status ftk_iso_plan_count(ftk_iso_plan *plan, int64_t *n) {
    if (n) *n = 0;
    if (!plan || !n) return fail(FTK_ERR_ARG, "plan and n must be non-NULL");
    ftk_status s = iso_settle(plan);
    if (s != FTK_OK) return s;
    *n = plan->h_ctr->edges;
    return FTK_OK;
}

ftk_status ftk_iso_plan_download(ftk_iso_plan *plan, ftk_iso_result **out) {
    if (out) *out = nullptr;
    if (!plan || !out) return fail(FTK_ERR_ARG, "plan and out must be non-NULL");
    ftk_status s = iso_settle(plan);
    if (s != FTK_OK) return s;
    return iso_download(plan, out);
}

ftk_status ftk_iso_plan_download_into(ftk_iso_plan *plan, ftk_iso_point *dst, int64_t cap, int64_t *n) {
    if (n) *n = 0;
    if (!plan || !n || (cap > 0 && !dst) || cap < 0) return fail(FTK_ERR_ARG, "invalid argument");
    ftk_status s = iso_settle(plan);
    if (s != FTK_OK) return s;
    const long long P = plan->h_ctr->edges;
    *n = P;
    if (P > cap) return fail(FTK_ERR_NOMEM, "the destination holds fewer records than the run produced");
    if (P > 0) {
        ISO_CUDA(cudaMemcpyAsync(dst, plan->W.rec, (size_t)P * sizeof(ftk_iso_point), cudaMemcpyDeviceToHost,
                                 plan->stream));
        ISO_CUDA(cudaStreamSynchronize(plan->stream));
    }
    return FTK_OK;
}

ftk_status ftk_iso_plan_device_records(ftk_iso_plan *plan, const ftk_iso_point **records, int64_t *n) {
    if (records) *records = nullptr;
    if (n) *n = 0;
    if (!plan || !records || !n) return fail(FTK_ERR_ARG, "invalid argument");
    ftk_status s = iso_settle(plan);
    if (s != FTK_OK) return s;
    *records = plan->W.rec;
    *n = plan->h_ctr->edges;
    return FTK_OK;
}

ftk_status ftk_iso_plan_stage_times(ftk_iso_plan *plan, float *ms, int cap, int *n) {
    if (n) *n = 0;
    if (!plan || !n || (cap > 0 && !ms)) return fail(FTK_ERR_ARG, "invalid argument");
    ftk_status s = iso_settle(plan);
    if (s != FTK_OK) return s;
    for (int i = 0; i < 4 && i < cap; ++i) ISO_CUDA(cudaEventElapsedTime(&ms[i], plan->ev[i], plan->ev[i + 1]));
    *n = std::min(cap, 4);
    return FTK_OK;
}

ftk_status ftk_iso_plan_destroy(ftk_iso_plan *plan) {
    if (!plan) return fail(FTK_ERR_ARG, "plan must be non-NULL");
    if (plan->executed) cudaStreamSynchronize(plan->stream);
    iso_destroy(plan);
    return FTK_OK;
}

static ftk_status iso_one_shot(int ndim, const float *f, int64_t nx, int64_t ny, int64_t nz, int64_t nt,
                               double isovalue, ftk_iso_result **out, void *cuda_stream) {
    if (out) *out = nullptr;
    if (!f || !out) return fail(FTK_ERR_ARG, "field and out must be non-NULL");
    ftk_iso_plan *pl = nullptr;
    ftk_status s = iso_create(ndim, nx, ny, nz, nt, &pl);
    if (s != FTK_OK) return s;
    s = iso_execute(pl, f, isovalue, (cudaStream_t)cuda_stream);
    if (s == FTK_OK) s = iso_settle(pl);
    if (s == FTK_OK) s = iso_download(pl, out);
    if (pl->executed) cudaStreamSynchronize(pl->stream);
    iso_destroy(pl);
    return s;
}

ftk_status ftk_track_iso2d(const float *f, int64_t nx, int64_t ny, int64_t nt, double isovalue,
                           ftk_iso_result **out, void *cuda_stream) {
    return iso_one_shot(2, f, nx, ny, 1, nt, isovalue, out, cuda_stream);
}

ftk_status ftk_track_iso3d(const float *f, int64_t nx, int64_t ny, int64_t nz, int64_t nt, double isovalue,
                           ftk_iso_result **out, void *cuda_stream) {
    return iso_one_shot(3, f, nx, ny, nz, nt, isovalue, out, cuda_stream);
}

size_t ftk_iso_result_count(const ftk_iso_result *r) { return r ? r->count : 0; }
const ftk_iso_point *ftk_iso_result_data(const ftk_iso_result *r) { return r ? r->data : nullptr; }
void ftk_iso_result_free(ftk_iso_result *r) {
    if (!r) return;
    std::free(r->data);
    delete r;
}

}  // extern "C"
