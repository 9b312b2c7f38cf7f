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
//   k_iso_pieces per owner whose unit cube lies in the grid: the cube's
//                cells (pentachora / tetrahedra, one per ordering of the
//                axes) unite their intersected edges in a small union-find
//                over the cube's 3^d - 2^d edge slots; each local piece is
//                represented by its smallest edge (global unions only for a
//                cube with several pieces); every edge records the
//                representative of its piece in its home cube.
//   k_iso_join   per such cube and axis: the pieces of two face-adjacent
//                cubes that share an intersected edge are united (lock-free
//                global union-find over edge indices).
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
    int small;           // every vertex id, edge id and item index < 2^31: FastDiv below
    FastDiv dW, dVC, dX, dY, dYZ, dE;   // by W, ceil(nx / 128), nx, ny, ny * nz, 2^d - 1
};

// n / d with the plan's fixed divisors (FastDiv when the grid is small)
__device__ __forceinline__ long long iso_div(const IsoGrid &G, long long n, const FastDiv &f, long long d) {
    return G.small ? (long long)fdiv((unsigned)n, f) : n / d;
}

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
    uint16_t *own_cb;              // [ocap] above bits of the corners of its unit cube
    int *own_rep;                  // [ocap] representative edge of its cube's piece (-1: several pieces)
    int *edge_rep;                 // [cap] representative of each edge's piece in its home cube
    const uint32_t *piece1;        // [2^(2^d) / 32] one-piece cube patterns (built with the plan)
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
    uint64_t elo[NC];   // slots 0-63 incident to corner c
    uint32_t ehi[NC];   // slot 64 (3D)
    __host__ __device__ constexpr IsoTables() : slot{}, sa{}, sb{}, chain{}, elo{}, ehi{} {
        int s = 0;
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) slot[a][b] = 255;
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b)
                if (a != b && (a & b) == a) {
                    slot[a][b] = (uint8_t)s;
                    sa[s] = (uint8_t)a;
                    sb[s] = (uint8_t)b;
                    if (s < 64) {
                        elo[a] |= 1ull << s;
                        elo[b] |= 1ull << s;
                    } else {
                        ehi[a] |= 1u;
                        ehi[b] |= 1u;
                    }
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

// For every cell and every above/below pattern of its d + 1 vertices (bit k
// = vertex k of the cell's chain above), the set of the cube's edge slots
// the cell intersects: the slots of its vertex pairs that disagree.
template <int N>
struct IsoCellMasks {
    static constexpr int D = N + 1, NCELL = IsoTables<N>::NCELL, NP = 1 << (D + 1);
    uint64_t lo[NCELL][NP];   // slots 0-63
    uint32_t hi[NCELL][NP];   // slot 64 (3D)
    __host__ __device__ constexpr IsoCellMasks() : lo{}, hi{} {
        const IsoTables<N> t;
        for (int p = 0; p < NCELL; ++p)
            for (int pat = 0; pat < NP; ++pat) {
                uint64_t l = 0;
                uint32_t h = 0;
                for (int i = 0; i <= D; ++i)
                    for (int j = i + 1; j <= D; ++j) {
                        if (((pat >> i) ^ (pat >> j)) & 1) {
                            const int sl = t.slot[t.chain[p][i]][t.chain[p][j]];
                            if (sl < 64) l |= 1ull << sl;
                            else h |= 1u;
                        }
                    }
                lo[p][pat] = l;
                hi[p][pat] = h;
            }
    }
};

__constant__ IsoTables<2> c_iso2 = IsoTables<2>();
__constant__ IsoTables<3> c_iso3 = IsoTables<3>();
template <int N> __device__ __forceinline__ const IsoTables<N> &iso_tables();
template <> __device__ __forceinline__ const IsoTables<2> &iso_tables<2>() { return c_iso2; }
template <> __device__ __forceinline__ const IsoTables<3> &iso_tables<3>() { return c_iso3; }
__constant__ IsoCellMasks<2> c_cmask2 = IsoCellMasks<2>();
__constant__ IsoCellMasks<3> c_cmask3 = IsoCellMasks<3>();
template <int N> __device__ __forceinline__ const IsoCellMasks<N> &iso_cell_masks();
template <> __device__ __forceinline__ const IsoCellMasks<2> &iso_cell_masks<2>() { return c_cmask2; }
template <> __device__ __forceinline__ const IsoCellMasks<3> &iso_cell_masks<3>() { return c_cmask3; }

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
// k_iso_bits: rows whose length is a multiple of 4 floats (and a 16-byte
// aligned field) take 16-byte loads -- lane l holds columns 4l .. 4l+3 of a
// 128-column chunk, eight lanes build one word from their 4-bit nibbles --
// other rows one float per lane.  A warp takes U consecutive items (chunks
// or words) per step and issues all their loads before any comparison.
// ---------------------------------------------------------------------------
template <bool VEC>
__global__ void __launch_bounds__(INT) k_iso_bits(IsoGrid G, IsoWork W) {
    constexpr int U = VEC ? 4 : 8;
    const int per_row = VEC ? (G.nx + 127) / 128 : G.W;   // items per row
    const long long items = G.rows * per_row;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * INT) >> 5;
    bool bad = false;
    for (long long it0 = (((long long)blockIdx.x * INT + threadIdx.x) >> 5) * U; it0 < items; it0 += nwarps * U) {
        long long row = iso_div(G, it0, VEC ? G.dVC : G.dW, per_row);
        int k = (int)(it0 - row * per_row);
        if (VEC) {
            float4 v[U];
            bool in[U];
            long long rw[U];
            int kk[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int x = k * 128 + lane * 4;
                in[u] = it0 + u < items && x < G.nx;
                v[u] = in[u] ? __ldg(reinterpret_cast<const float4 *>(G.f + row * G.nx + x)) : make_float4(0, 0, 0, 0);
                rw[u] = row;
                kk[u] = k;
                if (++k == per_row) {
                    k = 0;
                    ++row;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float4 a = v[u];
                bad |= in[u] && !(fabsf(a.x) <= FLT_MAX && fabsf(a.y) <= FLT_MAX && fabsf(a.z) <= FLT_MAX &&
                                  fabsf(a.w) <= FLT_MAX);
                uint32_t w = 0;
                if (in[u])
                    w = ((a.x >= G.c_up) | (a.y >= G.c_up) << 1 | (a.z >= G.c_up) << 2 | (a.w >= G.c_up) << 3)
                        << (4 * (lane & 7));
                w |= __shfl_xor_sync(ALL, w, 1);
                w |= __shfl_xor_sync(ALL, w, 2);
                w |= __shfl_xor_sync(ALL, w, 4);
                const int word = kk[u] * 4 + (lane >> 3);
                if ((lane & 7) == 0 && it0 + u < items && word < G.W) W.bits[rw[u] * G.W + word] = w;
            }
        } else {
            float v[U];
            bool in[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int x = k * 32 + lane;
                in[u] = it0 + u < items && x < G.nx;
                v[u] = in[u] ? __ldg(G.f + row * G.nx + x) : 0.0f;
                if (++k == per_row) {
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
    const long long t = iso_div(G, row, G.dYZ, ny * nz);
    const long long rz = row - t * ny * nz;
    const int z = (int)iso_div(G, rz, G.dY, ny), y = (int)(rz - (long long)z * ny);
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

// index (from 0) of the n-th set bit of m; n < popc(m)
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n) {
    int p = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (n >= c) {
            n -= c;
            m >>= w;
            p += w;
        }
    }
    return p;
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
    __shared__ uint32_t sX[E][INT];
    __shared__ uint32_t s_own[INT];
    __shared__ int s_wex[INT];
    __shared__ long long s_e0[INT], s_o0[INT], s_g0[INT];
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
            row = iso_div(G, it, G.dW, G.W);
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
        // the block's owners (vertices with an intersected edge of their
        // own) are handed out one per thread, in order: the item of owner j
        // is found among the items' exclusive owner counts, its vertex is
        // the rank-th set bit of the item's owner word, its first edge
        // follows the item's edges of the vertices left of it
#pragma unroll
        for (int m = 0; m < E; ++m) sX[m][threadIdx.x] = X[m];
        s_own[threadIdx.x] = own;
        s_e0[threadIdx.x] = e0;
        s_o0[threadIdx.x] = o0;
        s_g0[threadIdx.x] = row * G.nx + 32 * k;
        s_wex[threadIdx.x] = (int)(ex >> 31);   // owners of the tile before the item
        __syncthreads();
        const int btot = (int)(tot >> 31);
        for (int j = threadIdx.x; j < btot; j += INT) {
            int lo = 0, hi = INT - 1;   // last item whose exclusive count is <= j
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_wex[mid] <= j) lo = mid;
                else hi = mid - 1;
            }
            const int src = lo;
            const int r = j - s_wex[src];
            const uint32_t ow = s_own[src];
            const int b = nth_set_bit(ow, r);
            const uint32_t below = (1u << b) - 1u;
            uint32_t mask = 0;
            int pre = 0;
#pragma unroll
            for (int m = 1; m <= E; ++m) {
                const uint32_t xm = sX[m - 1][src];
                pre += __popc(xm & below);
                mask |= ((xm >> b) & 1u) << (m - 1);
            }
            long long e = s_e0[src] + pre;
            const long long oi = s_o0[src] + r;
            if (e + __popc(mask) > W.cap || oi >= W.ocap) {
                atomicOr(status, IST_OVERFLOW);
                continue;
            }
            const long long g = s_g0[src] + b;
            const float w0 = iso_w(__ldg(G.f + g), G.c_hi, G.c_lo);
            W.own_g[oi] = g;
            W.own_first[oi] = (int)e;
            W.own_mask[oi] = (uint16_t)mask;
#pragma unroll
            for (int m = 1; m <= E; ++m) {
                if (!((mask >> (m - 1)) & 1u)) continue;
                const float w1 = iso_w(__ldg(G.f + g + iso_step<N>(G, m)), G.c_hi, G.c_lo);
                const float den = w0 - w1;
                float mu = den != 0.0f ? w0 / den : 0.0f;
                mu = fminf(fmaxf(mu, 0.0f), 1.0f);
                W.id[e] = g * E + (m - 1);
                W.off[e] = make_float4((m & 1) ? mu : 0.0f, ((m >> 1) & 1) ? mu : 0.0f,
                                       N == 3 && ((m >> 2) & 1) ? mu : 0.0f, ((m >> N) & 1) ? mu : 0.0f);
                W.parent[e] = (int)e;
                W.edge_rep[e] = (int)e;
                ++e;
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

// unites x with the tree whose root was `root` (possibly stale); returns the
// root of the union (the smaller of the two roots)
__device__ __forceinline__ int iso_unite_root(int *parent, int x, int root, unsigned *status) {
    int a = iso_find(parent, x, status);
    int b = iso_find(parent, root, status);
    for (int it = 0; it < ISO_UF_LIMIT; ++it) {
        if (a == b) return a;
        if (a < b) { const int t = a; a = b; b = t; }
        const int old = atomicCAS(&parent[a], a, b);
        if (old == a) return b;
        a = iso_find(parent, old, status);
        b = iso_find(parent, b, status);
    }
    atomicOr(status, IST_TIMEOUT);
    return b;
}

// Cube of owner s: coordinates of its base vertex, whether the unit cube lies
// in the grid, and the axes along which it is the last cube (ub)
struct IsoCube {
    long long row;
    int x, y, z, t;
    bool inside;
    int ub;
};
template <int N>
__device__ __forceinline__ IsoCube iso_cube(const IsoGrid &G, long long g) {
    IsoCube q;
    q.row = iso_div(G, g, G.dX, G.nx);
    q.x = (int)(g - q.row * G.nx);
    const long long t = iso_div(G, q.row, G.dYZ, (long long)G.ny * G.nz);
    const long long rz = q.row - t * G.ny * G.nz;
    q.z = (int)iso_div(G, rz, G.dY, G.ny);
    q.y = (int)(rz - (long long)q.z * G.ny);
    q.t = (int)t;
    q.inside = q.x + 1 < G.nx && q.y + 1 < G.ny && (N != 3 || q.z + 1 < G.nz) && q.t + 1 < G.nt;
    q.ub = (q.x + 2 == G.nx ? 1 : 0) | (q.y + 2 == G.ny ? 2 : 0) | (N == 3 && q.z + 2 == G.nz ? 4 : 0) |
           (q.t + 2 == G.nt ? 1 << N : 0);
    return q;
}

// above bits of the cube's corners (bit a = corner a, a = axis mask)
template <int N>
__device__ __forceinline__ uint32_t iso_corners(const IsoGrid &G, const uint32_t *bits, const IsoCube &q) {
    constexpr int NC = 1 << (N + 1);
    uint32_t cb = 0;
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        const long long r2 = q.row + iso_row_step<N>(G, a);
        const int xa = q.x + (a & 1);
        cb |= ((bits[r2 * G.W + (xa >> 5)] >> (xa & 31)) & 1u) << a;
    }
    return cb;
}

// owner index of vertex (row, x): the item's owners before it plus the
// owners among the item's vertices left of it
__device__ __forceinline__ long long iso_owner(const IsoGrid &G, const IsoWork &W, long long row, int x) {
    const long long item = row * G.W + (x >> 5);
    return W.item_own[item] + __popc(W.obits[item] & ((1u << (x & 31)) - 1u));
}

// Local pieces of a unit cube with above bits cb: the intersected slot set
// of each cell (tables lo / hi by the cell's above/below pattern); sets that
// overlap belong to one piece, kept as up to K disjoint slot masks (many:
// more pieces than that); h* = every intersected slot.
template <int N, int K = 4>
__device__ __forceinline__ void iso_merge_cells(uint32_t cb, const uint64_t (*lo)[1 << (N + 2)],
                                                const uint32_t (*hi)[1 << (N + 2)], uint64_t (&clo)[K],
                                                uint32_t (&chi)[K], bool (&used)[K], bool &many, uint64_t &hlo,
                                                uint32_t &hhi) {
    using Tb = IsoTables<N>;
    constexpr int D = N + 1, NCELL = Tb::NCELL, NP = 1 << (D + 1);
    constexpr Tb TT{};   // the cell chains as compile-time constants of the unrolled loop
#pragma unroll
    for (int p = 0; p < NCELL; ++p) {
        int pat = 0;
#pragma unroll
        for (int k = 0; k <= D; ++k) pat |= ((cb >> TT.chain[p][k]) & 1) << k;
        if (pat == 0 || pat == NP - 1) continue;
        const uint64_t slo = lo[p][pat];
        const uint32_t shi = hi[p][pat];
        hlo |= slo;
        hhi |= shi;
        // merge every piece the cell's set touches into the first such
        int tgt = -1;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (!used[c] || !((clo[c] & slo) | (chi[c] & shi))) continue;
            if (tgt < 0) {
                tgt = c;
                clo[c] |= slo;
                chi[c] |= shi;
            }
        }
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (!used[c] || c == tgt || !((clo[c] & slo) | (chi[c] & shi))) continue;
#pragma unroll
            for (int d = 0; d < K; ++d)
                if (d == tgt) {
                    clo[d] |= clo[c];
                    chi[d] |= chi[c];
                }
            used[c] = false;
        }
        if (tgt < 0) {
            bool placed = false;
#pragma unroll
            for (int c = 0; c < K; ++c)
                if (!used[c] && !placed) {
                    used[c] = true;
                    clo[c] = slo;
                    chi[c] = shi;
                    placed = true;
                }
            many |= !placed;
        }
    }
}

// bit cb of piece1 = a unit cube whose corners have above bits cb holds one
// piece of the level set (one thread per pattern; 2^(2^d) patterns)
template <int N>
__global__ void __launch_bounds__(INT) k_iso_piece_table(uint32_t *piece1) {
    using Cm = IsoCellMasks<N>;
    constexpr int NCELL = IsoTables<N>::NCELL, NP = Cm::NP, NPAT = 1 << (1 << (N + 1));
    __shared__ uint64_t s_lo[NCELL][NP];
    __shared__ uint32_t s_hi[NCELL][NP];
    for (int i = threadIdx.x; i < NCELL * NP; i += INT) {
        s_lo[i / NP][i % NP] = iso_cell_masks<N>().lo[i / NP][i % NP];
        s_hi[i / NP][i % NP] = iso_cell_masks<N>().hi[i / NP][i % NP];
    }
    __syncthreads();
    const int cb = blockIdx.x * INT + threadIdx.x;
    bool one = false;
    if (cb < NPAT) {
        uint64_t clo[4] = {};
        uint32_t chi[4] = {};
        bool used[4] = {};
        bool many = false;
        uint64_t hlo = 0;
        uint32_t hhi = 0;
        iso_merge_cells<N>((uint32_t)cb, s_lo, s_hi, clo, chi, used, many, hlo, hhi);
        one = !many && (used[0] + used[1] + used[2] + used[3]) == 1;
    }
    const uint32_t w = __ballot_sync(ALL, one);
    if ((threadIdx.x & 31) == 0 && cb < NPAT) piece1[cb >> 5] = w;
}

// Cell pass, first kernel: one thread per owner whose unit cube lies in the
// grid.  Each cell of the cube intersects a set of the cube's edge slots
// (read from a table by the cell's above/below pattern); sets that overlap
// belong to one local piece, so the pieces are the unions of overlapping
// cell sets (kept as up to four disjoint slot masks).  Each piece is
// represented by its smallest edge index.  A cube with one piece (nearly
// every cube) stores that representative; a cube with several unites each
// edge with its piece's representative in the global union-find and stores
// -1 (more than four pieces: every cell's edges are united directly).  Every
// edge whose home cube this is -- the cube based at its lower vertex, or the
// last cube along an axis where that vertex is on the grid's upper face --
// records the representative of its piece.
template <int N>
__global__ void __launch_bounds__(INT, 2) k_iso_pieces(IsoGrid G, IsoWork W) {
    using Tb = IsoTables<N>;
    using Cm = IsoCellMasks<N>;
    constexpr int D = N + 1, NC = 1 << D, NS = Tb::NS, NCELL = Tb::NCELL, NP = Cm::NP;
    constexpr int K = 4;   // local pieces kept as masks
    __shared__ uint8_t s_sa[NS], s_sb[NS];
    __shared__ uint8_t s_chain[NCELL][D + 1];
    __shared__ uint64_t s_lo[NCELL][NP];
    __shared__ uint32_t s_hi[NCELL][NP];
    __shared__ int s_cf[NC][INT];        // per thread: first edge of each corner's owner
    __shared__ uint16_t s_cm[NC][INT];   // and its edge mask
    const int me = threadIdx.x;
    for (int i = threadIdx.x; i < NS; i += INT) {
        s_sa[i] = iso_tables<N>().sa[i];
        s_sb[i] = iso_tables<N>().sb[i];
    }
    for (int i = threadIdx.x; i < NCELL * (D + 1); i += INT)
        s_chain[i / (D + 1)][i % (D + 1)] = iso_tables<N>().chain[i / (D + 1)][i % (D + 1)];
    for (int i = threadIdx.x; i < NCELL * NP; i += INT) {
        s_lo[i / NP][i % NP] = iso_cell_masks<N>().lo[i / NP][i % NP];
        s_hi[i / NP][i % NP] = iso_cell_masks<N>().hi[i / NP][i % NP];
    }
    __syncthreads();
    if (W.ctr->status & (IST_OVERFLOW | IST_RANGE | IST_BIG)) return;
    const long long no = W.ctr->owners;
    unsigned *status = &W.ctr->status;
    for (long long s = blockIdx.x * (long long)INT + threadIdx.x; s < no; s += (long long)gridDim.x * INT) {
        const IsoCube q = iso_cube<N>(G, W.own_g[s]);
        if (!q.inside) continue;
        const uint32_t cb = iso_corners<N>(G, W.bits, q);
        W.own_cb[s] = (uint16_t)cb;
        const bool single = (W.piece1[cb >> 5] >> (cb & 31)) & 1u;
        uint64_t clo[K] = {};
        uint32_t chi[K] = {};
        bool used[K] = {};
        bool many = false;
        uint64_t hlo = 0;   // every intersected slot
        uint32_t hhi = 0;
        if (single) {
            // one piece: the intersected slots are those with exactly one
            // corner above, the XOR of the above corners' incidence masks
            constexpr Tb TT{};
#pragma unroll
            for (int a = 0; a < NC; ++a)
                if ((cb >> a) & 1u) {
                    hlo ^= TT.elo[a];
                    hhi ^= TT.ehi[a];
                }
            used[0] = true;
        } else {
            iso_merge_cells<N>(cb, s_lo, s_hi, clo, chi, used, many, hlo, hhi);
        }
        int npieces = 0;
#pragma unroll
        for (int c = 0; c < K; ++c) npieces += used[c];
        // edge indices through the owner lists of the edges' lower corners,
        // looked up for every such corner at once
        uint32_t need = 0;
        for (uint64_t r = hlo; r; r &= r - 1) need |= 1u << s_sa[__ffsll((long long)r) - 1];
        if (hhi) need |= 1u << s_sa[64];
        int cbase[NC];
        uint32_t cob[NC];
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            if (!((need >> a) & 1u)) continue;
            const int xa = q.x + (a & 1);
            const long long item = (q.row + iso_row_step<N>(G, a)) * G.W + (xa >> 5);
            cob[a] = W.obits[item] & ((1u << (xa & 31)) - 1u);
            cbase[a] = W.item_own[item];
        }
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            if (!((need >> a) & 1u)) continue;
            const long long o = cbase[a] + __popc(cob[a]);
            s_cf[a][me] = W.own_first[o];
            s_cm[a][me] = W.own_mask[o];
        }
        auto gidx = [&](int sl) -> int {
            const int a = s_sa[sl], m = a ^ s_sb[sl];
            return s_cf[a][me] + __popc((uint32_t)s_cm[a][me] & ((1u << (m - 1)) - 1u));
        };
        auto home = [&](int sl) -> bool { return !(s_sa[sl] & ~q.ub); };
        if (many) {
            // more local pieces than masks kept: every cell's edges united
            // directly; each edge represents itself
            W.own_rep[s] = -1;
#pragma unroll 1
            for (int p = 0; p < NCELL; ++p) {
                int pat = 0;
#pragma unroll
                for (int k = 0; k <= D; ++k) pat |= ((cb >> s_chain[p][k]) & 1) << k;
                if (pat == 0 || pat == NP - 1) continue;
                uint64_t slo = s_lo[p][pat];
                int first = -1;
                for (; slo; slo &= slo - 1) {
                    const int gi = gidx(__ffsll((long long)slo) - 1);
                    if (first < 0) first = gi;
                    else iso_unite_root(W.parent, gi, first, status);
                }
                if (s_hi[p][pat]) {
                    const int gi = gidx(64);
                    if (first >= 0) iso_unite_root(W.parent, gi, first, status);
                }
            }
            for (uint64_t r = hlo; r; r &= r - 1) {
                const int sl = __ffsll((long long)r) - 1;
                if (home(sl)) W.edge_rep[gidx(sl)] = gidx(sl);
            }
            if (hhi && home(64)) W.edge_rep[gidx(64)] = gidx(64);
            continue;
        }
        if (npieces == 1) {
            int rep = INT32_MAX;
            for (uint64_t r = hlo; r; r &= r - 1) rep = min(rep, gidx(__ffsll((long long)r) - 1));
            if (hhi) rep = min(rep, gidx(64));
            W.own_rep[s] = rep;
            for (uint64_t r = hlo; r; r &= r - 1) {
                const int sl = __ffsll((long long)r) - 1;
                if (home(sl)) W.edge_rep[gidx(sl)] = rep;
            }
            if (hhi && home(64)) W.edge_rep[gidx(64)] = rep;
            continue;
        }
        // several pieces: the smallest edge index of each, then every edge
        // united with it
        W.own_rep[s] = -1;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (!used[c]) continue;
            int rep = INT32_MAX;
            for (uint64_t r = clo[c]; r; r &= r - 1) rep = min(rep, gidx(__ffsll((long long)r) - 1));
            if (chi[c]) rep = min(rep, gidx(64));
            for (uint64_t r = clo[c]; r; r &= r - 1) {
                const int sl = __ffsll((long long)r) - 1;
                const int gi = gidx(sl);
                if (gi != rep) iso_unite_root(W.parent, gi, rep, status);
                if (home(sl)) W.edge_rep[gi] = rep;
            }
            if (chi[c]) {
                const int gi = gidx(64);
                if (gi != rep) iso_unite_root(W.parent, gi, rep, status);
                if (home(64)) W.edge_rep[gi] = rep;
            }
        }
    }
}

// Cell pass, second kernel: one thread per owner whose cube lies in the
// grid.  For each axis a with a next cube along a, if the common face has
// intersected edges the two cubes' pieces through them are joined: two
// one-piece cubes unite their representatives; a one-piece cube and a
// several-piece cube unite the representative with each shared intersected
// edge (the other cube has united those with its own pieces).  The cubes
// holding any one edge are joined face to face through cubes that all hold
// it, so this connects every pair of pieces that share an edge.
template <int N>
__global__ void __launch_bounds__(INT) k_iso_join(IsoGrid G, IsoWork W) {
    using Tb = IsoTables<N>;
    constexpr int D = N + 1, NC = 1 << D, NS = Tb::NS;
    __shared__ uint8_t s_sa[NS], s_sb[NS];
    for (int i = threadIdx.x; i < NS; i += INT) {
        s_sa[i] = iso_tables<N>().sa[i];
        s_sb[i] = iso_tables<N>().sb[i];
    }
    __syncthreads();
    if (W.ctr->status & (IST_OVERFLOW | IST_RANGE | IST_BIG)) return;
    const long long no = W.ctr->owners;
    unsigned *status = &W.ctr->status;
    for (long long s = blockIdx.x * (long long)INT + threadIdx.x; s < no; s += (long long)gridDim.x * INT) {
        const IsoCube q = iso_cube<N>(G, W.own_g[s]);
        if (!q.inside) continue;
        const uint32_t cb = W.own_cb[s];
        const int rep = W.own_rep[s];
        int cur = rep;   // root of rep's tree after the unions so far
        // the next cube along each axis whose common face has an intersected
        // edge (its base vertex then owns one): all looked up at once
        uint32_t act = 0;
        int rep2s[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            uint32_t fm = 0;                          // corners on the face x_a = +1
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if ((c >> a) & 1) fm |= 1u << c;
            const uint32_t fc = cb & fm;
            if (!((q.ub >> a) & 1) && fc != 0 && fc != fm) act |= 1u << a;
        }
        long long nown[D];
#pragma unroll
        for (int a = 0; a < D; ++a)
            if ((act >> a) & 1) nown[a] = iso_owner(G, W, q.row + iso_row_step<N>(G, 1 << a), q.x + (a == 0));
#pragma unroll
        for (int a = 0; a < D; ++a)
            if ((act >> a) & 1) rep2s[a] = W.own_rep[nown[a]];
#pragma unroll 1
        for (int a = 0; a < D; ++a) {
            if (!((act >> a) & 1)) continue;
            int rep2 = 0;
#pragma unroll
            for (int b = 0; b < D; ++b)
                if (b == a) rep2 = rep2s[b];
            if (rep >= 0 && rep2 >= 0) {
                cur = iso_unite_root(W.parent, rep2, cur, status);
                continue;
            }
            if (rep < 0 && rep2 < 0) continue;
            // one side has several pieces: unite the other side's
            // representative with every intersected edge of the face
            const int one = rep >= 0 ? rep : rep2;
            for (int sl = 0; sl < NS; ++sl) {
                const int ca = s_sa[sl], cbb = s_sb[sl];
                if (!((ca >> a) & 1) || !(((cb >> ca) ^ (cb >> cbb)) & 1u)) continue;   // sb has bit a too
                const int xa = q.x + (ca & 1);
                const long long o = iso_owner(G, W, q.row + iso_row_step<N>(G, ca), xa);
                const int m = ca ^ cbb;
                const int e = W.own_first[o] + __popc((uint32_t)W.own_mask[o] & ((1u << (m - 1)) - 1u));
                iso_unite_root(W.parent, e, one, status);
            }
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
    // a block's records are built in shared memory and stored as one
    // contiguous run of 16-byte words (INT records of 56 bytes start on a
    // 16-byte boundary)
    static_assert(sizeof(ftk_iso_point) == 56 && (INT * sizeof(ftk_iso_point)) % 16 == 0, "record layout");
    __shared__ __align__(16) ftk_iso_point recs[INT];
    if (W.ctr->status & (IST_OVERFLOW | IST_RANGE | IST_BIG)) return;
    const long long P = W.ctr->edges;
    unsigned *status = &W.ctr->status;
    for (long long i0 = blockIdx.x * (long long)INT; i0 < P; i0 += (long long)gridDim.x * INT) {
        const long long i = i0 + threadIdx.x;
        if (i < P) {
            const int r = iso_find(W.parent, W.edge_rep[i], status);
            const long long id = W.id[i];
            const long long g = iso_div(G, id, G.dE, E);
            const int m = (int)(id - g * E) + 1;
            const long long row = iso_div(G, g, G.dX, G.nx);
            const int x = (int)(g - row * G.nx);
            const long long tt = iso_div(G, row, G.dYZ, (long long)G.ny * G.nz);
            const long long rz = row - tt * G.ny * G.nz;
            const int z = (int)iso_div(G, rz, G.dY, G.ny), y = (int)(rz - (long long)z * G.ny);
            ftk_iso_point &p = recs[threadIdx.x];
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
        }
        __syncthreads();
        const long long n = P - i0 < INT ? P - i0 : INT;
        const int nbytes = (int)n * (int)sizeof(ftk_iso_point);
        const uint4 *src = reinterpret_cast<const uint4 *>(recs);
        uint4 *dst = reinterpret_cast<uint4 *>(W.rec + i0);
        for (int k = threadIdx.x; k < nbytes / 16; k += INT) dst[k] = src[k];
        if ((nbytes & 15) && threadIdx.x == 0) {   // odd count: the last 8 bytes
            const int k = nbytes / 8 - 1;
            reinterpret_cast<unsigned long long *>(W.rec + i0)[k] = reinterpret_cast<const unsigned long long *>(recs)[k];
        }
        __syncthreads();
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

// ---- host side: plans and the C ABI ----
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
    cudaFree(W.own_cb);
    cudaFree(W.own_rep);
    cudaFree(W.edge_rep);
    cudaFree(W.id);
    cudaFree(W.off);
    cudaFree(W.parent);
    cudaFree(W.rec);
    W.own_g = nullptr;
    W.own_first = nullptr;
    W.own_mask = nullptr;
    W.own_cb = nullptr;
    W.own_rep = nullptr;
    W.edge_rep = nullptr;
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
        cudaMalloc(&W.own_cb, sizeof(uint16_t) * ocap) != cudaSuccess ||
        cudaMalloc(&W.own_rep, sizeof(int) * ocap) != cudaSuccess ||
        cudaMalloc(&W.edge_rep, sizeof(int) * cap) != cudaSuccess ||
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
    cudaFree(const_cast<uint32_t *>(pl->W.piece1));
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
    // 16-byte loads when every row starts on a 16-byte boundary
    const bool vec = pl->G.nx % 4 == 0 && (reinterpret_cast<uintptr_t>(dev_f) & 15) == 0;
    const long long bitems = vec ? pl->G.rows * ((pl->G.nx + 127) / 128) : items;
    const unsigned gb = (unsigned)std::max<long long>(1, std::min<long long>((bitems + 31) / 32, (long long)sms * 8));
    ISO_CUDA(cudaEventRecord(pl->ev[0], s));
    if (vec) k_iso_bits<true><<<gb, INT, 0, s>>>(pl->G, W);
    else k_iso_bits<false><<<gb, INT, 0, s>>>(pl->G, W);
    ISO_CUDA(cudaEventRecord(pl->ev[1], s));
    const unsigned ge = (unsigned)std::max<long long>(1, std::min<long long>(pl->ntiles, (long long)sms * 4));
    const unsigned gl = (unsigned)std::max<long long>(1, std::min<long long>((W.ocap + INT - 1) / INT, (long long)sms * 8));
    const unsigned gL = (unsigned)std::max<long long>(1, std::min<long long>((W.cap + INT - 1) / INT, (long long)sms * 8));
    if (pl->ndim == 2) {
        k_iso_emit<2><<<ge, INT, 0, s>>>(pl->G, W);
        ISO_CUDA(cudaEventRecord(pl->ev[2], s));
        k_iso_pieces<2><<<gl, INT, 0, s>>>(pl->G, W);
        k_iso_join<2><<<gl, INT, 0, s>>>(pl->G, W);
        ISO_CUDA(cudaEventRecord(pl->ev[3], s));
        k_iso_label<2><<<gL, INT, 0, s>>>(pl->G, W);
    } else {
        k_iso_emit<3><<<ge, INT, 0, s>>>(pl->G, W);
        ISO_CUDA(cudaEventRecord(pl->ev[2], s));
        k_iso_pieces<3><<<gl, INT, 0, s>>>(pl->G, W);
        k_iso_join<3><<<gl, INT, 0, s>>>(pl->G, W);
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
    const int E = (1 << (ndim + 1)) - 1;
    G.small = (double)pl->nverts * E < 2147483648.0 ? 1 : 0;
    G.dW = make_fastdiv((unsigned)G.W);
    G.dVC = make_fastdiv((unsigned)((nx + 127) / 128));
    G.dX = make_fastdiv((unsigned)nx);
    G.dY = make_fastdiv((unsigned)ny);
    G.dYZ = make_fastdiv((unsigned)(ny * nz <= INT32_MAX ? ny * nz : 1));
    G.dE = make_fastdiv((unsigned)E);
    if (ny * nz > INT32_MAX) G.small = 0;
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
    {
        // the one-piece cube patterns, computed once for the plan
        const int npat = 1 << (1 << (ndim + 1));
        uint32_t *tab = nullptr;
        if (cudaMalloc(&tab, sizeof(uint32_t) * (npat / 32)) != cudaSuccess)
            return bad("device allocation of the piece table failed");
        W.piece1 = tab;
        if (ndim == 2) k_iso_piece_table<2><<<(npat + INT - 1) / INT, INT>>>(tab);
        else k_iso_piece_table<3><<<(npat + INT - 1) / INT, INT>>>(tab);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess)
            return bad("the piece table kernel failed");
    }
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
