// CUDA kernels of the exact critical-point tracking pipeline (sm_103a).
//
// Two forms of paper Algorithm 1 (left column, with Sec. 4.1 / 4.3).
//
// Streaming variants (the default; the dense pass is k_detect2_stream in
// ftk_detect2.cu and k_detect3_stream in ftk_detect3.cu):
//   detect       dense, HBM-bound: stream the field once, quantise
//                F = rint(f 2^S), integer central-difference gradient, and
//                cull every spacetime cube exactly -- a gradient component
//                that is < 0 on every corner, or >= 0 on every corner, rules
//                out every face owned by the cube (the symbolic perturbation
//                is infinitesimal and adds a positive term to a zero
//                component).  Surviving cubes are listed per segment
//                (t, z, y-block) in vertex order.
//   k_survive_eval  exact SoS predicate on every face of a surviving cube:
//                a mask of punctured face types.
//   k_survive_scan  global exclusive scan of the masks' popcounts.
//   k_seg_scan   segment totals and offsets in face-id order (look-back scan).
//   k_emit       punctured faces written at their sorted positions.
//   k_locate     location from the barycentric coordinates of Eq. (1) (FP32)
//                and Morse index of the interpolated Hessian (exact;
//                floating-point filters decide where they can certify).
//   k_link_survivors  per surviving cube: the cells it holds, each joining
//                its two punctured sides (lock-free union-find).
//   k_label      label = smallest face id of the component; pack records.
//
// Tiled variant (a fallback for rows the streaming kernels do not take):
//   k_detect     per unit: cull, exact predicate and compaction in one kernel.
//   k_scan       exclusive scan of the per-segment counts.
//   k_finalize   per puncture: rank, location, Morse index.
//   k_link       per puncture: its <= 2 cells, the other punctured side of
//                each (binary search), union-find.
//   k_label      as above.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <mutex>

#include "ftk_device.cuh"
#include "ftk_kernels.cuh"
#include "ftk_sparse.cuh"
#include "ftk_tma.cuh"

namespace ftk {

__constant__ MeshTables<2> c_mesh2 = MeshTables<2>();
__constant__ MeshTables<3> c_mesh3 = MeshTables<3>();

template <int N> __device__ __forceinline__ const MeshTables<N> &mesh();
template <> __device__ __forceinline__ const MeshTables<2> &mesh<2>() { return c_mesh2; }
template <> __device__ __forceinline__ const MeshTables<3> &mesh<3>() { return c_mesh3; }
__constant__ CellTables<2> c_cell2 = CellTables<2>();
__constant__ CellTables<3> c_cell3 = CellTables<3>();
template <int N> __device__ __forceinline__ const CellTables<N> &cells();
template <> __device__ __forceinline__ const CellTables<2> &cells<2>() { return c_cell2; }
template <> __device__ __forceinline__ const CellTables<3> &cells<3>() { return c_cell3; }

constexpr int NT = 256;              // threads per CTA of every kernel here
constexpr int UF_LIMIT = 1 << 22;    // bound on union-find retries / path steps
// The bounds in force, set from the host so that a test can make a bounded
// loop run out (the mbarrier waits of the detect kernels, which also drain
// copies in flight, keep their own fixed bound): the look-back bound in
// constant memory (read once per tile)
__constant__ long long g_lookback_cycles = WAIT_CYCLES;
// the union-find bound of the label pass, handed to each launch as a kernel
// parameter (Workspace::uf_limit); the pass takes it only in the instance a
// test selects, so that the normal instance keeps a compile-time bound
static std::atomic<int> g_host_uf_limit{UF_LIMIT};

// Exact SoS puncture test of one face; V[k] = gradient at the k-th vertex in
// increasing global-id order.
template <int N>
__device__ bool face_punctured(const int32_t (&V)[N + 1][N]) {
    // a component that is < 0 on every vertex, or >= 0 on every vertex,
    // excludes the origin: SoS perturbs a zero entry by a positive
    // infinitesimal, so zero counts as positive
#pragma unroll
    for (int r = 0; r < N; ++r) {
        bool allp = true, alln = true;
#pragma unroll
        for (int k = 0; k <= N; ++k) {
            allp &= V[k][r] >= 0;
            alln &= V[k][r] < 0;
        }
        if (allp || alln) return false;
    }
    int ref = 0;
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        int32_t M[N][N];
        int c = 0;
#pragma unroll
        for (int j = 0; j <= N; ++j) {
            if (j == k) continue;
#pragma unroll
            for (int r = 0; r < N; ++r) M[c][r] = V[j][r];
            ++c;
        }
        const int s = sos_det_sign<N>(M);
        const int val = (k & 1) ? -s : s;
        if (k == 0) ref = val;
        else if (val != ref) return false;
    }
    return true;
}

// ----------------------------------------------------------------------------
// Block-wide exclusive scan (NT threads); red needs NT/32 + 1 ints.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *red, T &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NT / 32 ? red[lane] : T(0);
#pragma unroll
        for (int o = 1; o < NT / 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) red[lane] = w;
    }
    __syncthreads();
    const T before = warp ? red[warp - 1] : T(0);
    total = red[NT / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// ----------------------------------------------------------------------------
// Single-pass scan across tiles by decoupled look-back (Merrill & Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016).  A tile
// publishes its total as soon as it is known, then walks back over its
// predecessors 32 at a time, summing their totals until one of them has
// published its inclusive prefix.  Tiles are numbered in the order blocks
// claim them, so every predecessor belongs to a running or finished block.
// State word: bits 62-63 = 1 (total) or 2 (inclusive prefix), bits 0-61 =
// the value; 0 = nothing yet.  The payload travels in the flag's own word,
// so plain volatile accesses suffice.  Called by one full warp; returns the
// exclusive prefix of tile t on every lane.
// ----------------------------------------------------------------------------
constexpr unsigned long long LB_AGG = 1ull << 62, LB_INC = 2ull << 62, LB_VAL = (1ull << 62) - 1;

__device__ long long warp_lookback(unsigned long long *tile_state, long long t, long long total,
                                   unsigned *status) {
    volatile unsigned long long *st = tile_state;
    const int lane = threadIdx.x & 31;
    if (lane == 0) st[t] = (t == 0 ? LB_INC : LB_AGG) | (unsigned long long)total;
    if (t == 0) return 0;
    long long ex = 0;
    long long hi = t - 1;   // highest predecessor not yet summed
    const long long t0 = clock64();
    while (true) {
        const long long j = hi - lane;
        unsigned long long v = LB_INC;   // before tile 0: prefix 0
        if (j >= 0) v = st[j];
        if (__any_sync(0xffffffffu, (v >> 62) == 0)) {
            if (clock64() - t0 > g_lookback_cycles) {
                if (lane == 0) atomicOr(status, ST_TIMEOUT);
                break;
            }
            __nanosleep(32);
            continue;
        }
        const unsigned inc = __ballot_sync(0xffffffffu, (v >> 62) == 2);
        const int stop = inc ? __ffs(inc) - 1 : 31;
        long long x = lane <= stop ? (long long)(v & LB_VAL) : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        ex += x;
        if (inc) break;
        hi -= 32;
    }
    if (lane == 0) st[t] = LB_INC | (unsigned long long)(ex + total);
    return ex;
}

// ----------------------------------------------------------------------------
// Detect kernel
// ----------------------------------------------------------------------------
struct TileGeom {
    int nx, ny, nz;
    int x0, y0, z0;
    int ncx, nvx;   // cubes and word columns of the unit's x window (from x0)
    int tw, ww;     // tile and word row strides: tile column j is x0 - 1 + j, word column j is x0 + j
    int PY, PZ;     // tile rows / planes (with halo)
    int WY, WZ;     // word rows / planes
    int tile;       // ints per F tile
    int wtile;      // bytes per word tile
    int vec;        // 1: the tile holds a 2D vector per vertex (the vectors are the "gradients")
};

__device__ __forceinline__ int quantise(float f, float scale, unsigned *status) {
    const float v = f * scale;   // exact: scale is a power of two
    if (!(fabsf(v) <= RANGE_LIMIT)) {
        atomicOr(status, ST_RANGE);
        return 0;
    }
    return __float2int_rn(v);
}

// gradient at (x, y, z) from an F tile; ty/tz are the tile row/plane of (y, z)
template <int N>
__device__ __forceinline__ void grad_tile(const int32_t *T, const TileGeom &g, int x, int y, int z,
                                          int ty, int tz, int32_t (&G)[N]) {
    const int lx = x - g.x0 + 1;    // tile column of x
    if (N == 2 && g.vec) {
        // a vector field: the quantised vector itself takes the gradient's place
        const int32_t *p = T + ((tz * g.PY + ty) * g.tw + lx) * 2;
        G[0] = p[0];
        G[1] = p[1];
        return;
    }
    const int32_t *row = T + (tz * g.PY + ty) * g.tw;
    G[0] = x == 0 ? 2 * (row[lx + 1] - row[lx])
         : x == g.nx - 1 ? 2 * (row[lx] - row[lx - 1])
         : row[lx + 1] - row[lx - 1];
    const int32_t *up = row + g.tw, *dn = row - g.tw;
    G[1] = y == 0 ? 2 * (up[lx] - row[lx])
         : y == g.ny - 1 ? 2 * (row[lx] - dn[lx])
         : up[lx] - dn[lx];
    if (N == 3) {
        const int ps = g.PY * g.tw;
        const int32_t *fw = row + ps, *bk = row - ps;
        G[N - 1] = z == 0 ? 2 * (fw[lx] - row[lx])
                 : z == g.nz - 1 ? 2 * (row[lx] - bk[lx])
                 : fw[lx] - bk[lx];
    }
}

template <int N>
__device__ void load_tile(const Field &F, const TileGeom &g, int s, int32_t *T, unsigned *status) {
    const int rows = g.PZ * g.PY;
    // samples of the window's cubes and their gradients' neighbours
    const int xlo = max(g.x0 - 1, 0), xhi = min(g.nx, g.x0 + g.ncx + 2);
    for (int i = threadIdx.x; i < rows * g.tw; i += NT) {
        const int x = g.x0 - 1 + i % g.tw;
        const int r = i / g.tw;
        const int ty = r % g.PY;
        const int tz = r / g.PY;
        const int y = g.y0 - 1 + ty;
        const int z = N == 3 ? g.z0 - 1 + tz : 0;
        if (x < xlo || x >= xhi || y < 0 || y >= g.ny || z < 0 || z >= g.nz) continue;
        const long long idx = (((long long)s * g.nz + z) * g.ny + y) * F.pitch + x;
        if (N == 2 && g.vec) {
            T[2 * i] = quantise(__ldg(F.f + 2 * idx), F.scale, status);
            T[2 * i + 1] = quantise(__ldg(F.f + 2 * idx + 1), F.scale, status);
        } else {
            T[i] = quantise(__ldg(F.f + idx), F.scale, status);
        }
    }
}

template <int N>
__device__ void make_words(const TileGeom &g, const int32_t *T, uint8_t *Wd) {
    for (int i = threadIdx.x; i < g.WZ * g.WY * g.nvx; i += NT) {
        const int j = i % g.nvx;
        const int x = g.x0 + j;
        const int r = i / g.nvx;
        const int wy = r % g.WY;
        const int wz = r / g.WY;
        const int y = g.y0 + wy;
        const int z = g.z0 + wz;
        if (y >= g.ny || z >= g.nz) continue;
        int32_t G[N];
        grad_tile<N>(T, g, x, y, z, wy + 1, N == 3 ? wz + 1 : 0, G);
        uint32_t w = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) w |= ((uint32_t)(G[c] < 0) << (2 * c)) | ((uint32_t)(G[c] >= 0) << (2 * c + 1));
        Wd[r * g.ww + j] = (uint8_t)w;
    }
}

template <int N>
__device__ __forceinline__ bool eval_face(const TileGeom &g, const int32_t *T0, const int32_t *T1,
                                          bool has_next, int x, int y, int z, int ly, int lz, int tt) {
    constexpr int TB = MeshDims<N>::TBIT;
    const uint8_t *ch = mesh<N>().face[tt];
    const int last = ch[N - 1];
    if ((last & 1) && x + 1 >= g.nx) return false;
    if ((last & 2) && y + 1 >= g.ny) return false;
    if (N == 3 && (last & 4) && z + 1 >= g.nz) return false;
    if ((last & TB) && !has_next) return false;
    int32_t V[N + 1][N];
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        const int m = k == 0 ? 0 : ch[k - 1];
        const int dx = m & 1, dy = (m >> 1) & 1, dz = N == 3 ? (m >> 2) & 1 : 0;
        const int32_t *T = (m & TB) ? T1 : T0;
        grad_tile<N>(T, g, x + dx, y + dy, z + dz, ly + dy + 1, N == 3 ? lz + dz + 1 : 0, V[k]);
    }
    return face_punctured<N>(V);
}

__host__ __device__ inline int round_up16(int v) { return (v + 15) & ~15; }

struct DetectLayout {
    int tile, wtile, plane_bits, plane_words, flag_words;
    int off_words, off_bm, off_sv, off_flags, off_red, total;
};

template <int N>
__host__ __device__ inline DetectLayout detect_layout(int wx, int ry, int rz, int comps = 1) {
    // wx: cube columns per unit (the row, or its window); the tile holds
    // wx + 3 sample columns (one left of the window, two right), the word
    // tile wx + 1
    DetectLayout L;
    const int PY = ry + 3, PZ = N == 3 ? rz + 3 : 1;
    const int WY = ry + 1, WZ = N == 3 ? rz + 1 : 1;
    const int RZ = N == 3 ? rz : 1;
    L.tile = (comps == 2 ? 2 : 1) * PZ * PY * (wx + 3);
    L.wtile = WZ * WY * (wx + 1);
    L.plane_bits = ry * wx;
    L.plane_words = (L.plane_bits + 31) / 32;
    L.flag_words = (L.plane_bits * MeshDims<N>::T + 31) / 32;
    L.off_words = 2 * L.tile * 4;
    L.off_bm = round_up16(L.off_words + 2 * L.wtile);
    L.off_sv = round_up16(L.off_bm + RZ * L.plane_words * 4);
    L.off_flags = round_up16(L.off_sv + L.plane_bits * 4);
    L.off_red = round_up16(L.off_flags + L.flag_words * 4);
    L.total = round_up16(L.off_red + 64 * 8);
    return L;
}

template <int N>
__global__ void __launch_bounds__(NT) k_detect(Field F, Blocking B, Workspace W) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int T = MeshDims<N>::T;
    const int rz = N == 3 ? B.rz : 1;
    const int wx = B.nxb > 1 ? B.wx : F.nx;
    const DetectLayout L = detect_layout<N>(wx, B.ry, B.rz, F.comps);
    int32_t *Ft = reinterpret_cast<int32_t *>(smem);
    uint8_t *Wt = smem + L.off_words;
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem + L.off_bm);
    int *sv = reinterpret_cast<int *>(smem + L.off_sv);
    uint32_t *flags = reinterpret_cast<uint32_t *>(smem + L.off_flags);
    long long *red = reinterpret_cast<long long *>(smem + L.off_red);
    __shared__ long long s_base;

    int u = blockIdx.x;
    const int tci = u % B.ntc;
    u /= B.ntc;
    const int nxb = B.nxb > 1 ? B.nxb : 1;
    const int xb = u % nxb;
    u /= nxb;
    const int yb = u % B.nyb;
    const int zb = u / B.nyb;

    TileGeom g;
    g.nx = F.nx; g.ny = F.ny; g.nz = F.nz;
    g.x0 = xb * wx;
    g.ncx = min(F.nx - g.x0, wx);
    g.nvx = min(F.nx - g.x0, g.ncx + 1);
    g.tw = wx + 3;
    g.ww = wx + 1;
    g.y0 = yb * B.ry;
    g.z0 = N == 3 ? zb * B.rz : 0;
    g.PY = B.ry + 3; g.PZ = N == 3 ? B.rz + 3 : 1;
    g.WY = B.ry + 1; g.WZ = N == 3 ? B.rz + 1 : 1;
    g.tile = L.tile; g.wtile = L.wtile;
    g.vec = F.comps == 2 ? 1 : 0;

    const int t_begin = tci * B.tc;
    const int t_end = min(F.nt, t_begin + B.tc);
    unsigned *status = &W.ctr->status;

    load_tile<N>(F, g, t_begin, Ft, status);
    __syncthreads();
    make_words<N>(g, Ft, Wt);
    int cur = 0;
    for (int t = t_begin; t < t_end; ++t) {
        const bool has_next = t + 1 < F.nt;
        const int nxt = cur ^ 1;
        const int32_t *T0 = Ft + cur * L.tile;
        const int32_t *T1 = Ft + nxt * L.tile;
        if (has_next) {
            load_tile<N>(F, g, t + 1, Ft + nxt * L.tile, status);
            __syncthreads();
            make_words<N>(g, T1, Wt + nxt * L.wtile);
        }
        for (int i = threadIdx.x; i < rz * L.plane_words; i += NT) bm[i] = 0u;
        __syncthreads();

        // ---- exact cube cull ------------------------------------------------
        bool any = false;
        for (int i = threadIdx.x; i < rz * B.ry * g.ncx; i += NT) {
            const int j = i % g.ncx;
            const int x = g.x0 + j;
            const int r = i / g.ncx;
            const int ly = r % B.ry;
            const int lz = r / B.ry;
            const int y = g.y0 + ly, z = g.z0 + lz;
            if (y >= g.ny || z >= g.nz) continue;
            const int ex = x + 1 < g.nx, ey = y + 1 < g.ny, ez = (N == 3) && (z + 1 < g.nz);
            uint32_t m = 0xffu;
            for (int ds = 0; ds <= (int)has_next; ++ds) {
                const uint8_t *wb = Wt + (cur ^ ds) * L.wtile;
                for (int dz = 0; dz <= ez; ++dz)
                    for (int dy = 0; dy <= ey; ++dy) {
                        const uint8_t *wr = wb + ((lz + dz) * g.WY + ly + dy) * g.ww + j;
                        m &= wr[0];
                        if (ex) m &= wr[1];
                    }
            }
            if (m == 0u) {
                const int idx = ly * g.ncx + j;
                atomicOr(&bm[lz * L.plane_words + (idx >> 5)], 1u << (idx & 31));
                any = true;
            }
        }
        const int any_all = __syncthreads_or(any);

        // ---- survivors: exact predicate, ordered compaction per segment -----
        for (int lz = 0; lz < rz; ++lz) {
            const int z = g.z0 + lz;
            if (z >= g.nz) break;
            const long long seg = (((long long)t * g.nz + z) * B.nyb + yb) * nxb + xb;
            if (!any_all) {
                if (threadIdx.x == 0) { W.seg_cnt[seg] = 0; W.seg_stage[seg] = 0; }
                continue;
            }
            // survivor list in vertex order
            int nsv = 0;
            for (int b0 = 0; b0 < L.plane_words; b0 += NT) {
                const int i = b0 + threadIdx.x;
                uint32_t bits = i < L.plane_words ? bm[lz * L.plane_words + i] : 0u;
                long long tot;
                long long pos = nsv + block_excl_scan<long long>(__popc(bits), red, tot);
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    sv[pos++] = i * 32 + b;
                }
                nsv += (int)tot;
            }
            const int ncand = nsv * T;
            const int nfw = (ncand + 31) / 32;
            for (int i = threadIdx.x; i < nfw; i += NT) flags[i] = 0u;
            __syncthreads();
            for (int c = threadIdx.x; c < ncand; c += NT) {
                const int v = sv[c / T];
                const int tt = c % T;
                const int ly = v / g.ncx, x = g.x0 + v % g.ncx;
                if (eval_face<N>(g, T0, T1, has_next, x, g.y0 + ly, z, ly, lz, tt))
                    atomicOr(&flags[c >> 5], 1u << (c & 31));
            }
            __syncthreads();
            long long mine = 0;
            for (int i = threadIdx.x; i < nfw; i += NT) mine += __popc(flags[i]);
            long long count;
            block_excl_scan<long long>(mine, red, count);
            if (threadIdx.x == 0) {
                const long long base = count ? (long long)atomicAdd(&W.ctr->staged, (unsigned long long)count) : 0;
                W.seg_cnt[seg] = (int)count;
                W.seg_stage[seg] = base;
                s_base = base;
                if (base + count > W.cap) atomicOr(status, ST_OVERFLOW);
            }
            __syncthreads();
            const long long base = s_base;
            long long run = 0;
            for (int b0 = 0; b0 < nfw; b0 += NT) {
                const int i = b0 + threadIdx.x;
                uint32_t bits = i < nfw ? flags[i] : 0u;
                long long tot;
                long long pos = base + run + block_excl_scan<long long>(__popc(bits), red, tot);
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int c = i * 32 + b;
                    const int v = sv[c / T];
                    const int ly = v / g.ncx, x = g.x0 + v % g.ncx;
                    const long long gid = (((long long)t * g.nz + z) * g.ny + g.y0 + ly) * g.nx + x;
                    if (pos < W.cap) W.staging[pos] = gid * T + (c % T);
                    ++pos;
                }
                run += tot;
            }
            __syncthreads();
        }
        __syncthreads();
        cur = nxt;
    }
}

// ----------------------------------------------------------------------------
// Scan of per-segment counts (one CTA)
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_scan(Workspace W) {
    __shared__ long long red[NT / 32 + 1];
    constexpr int PER = 16;
    long long run = 0;
    for (long long b0 = 0; b0 < W.nseg; b0 += (long long)NT * PER) {
        const long long i0 = b0 + (long long)threadIdx.x * PER;
        long long loc[PER];
        long long s = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const long long i = i0 + j;
            loc[j] = i < W.nseg ? (long long)W.seg_cnt[i] : 0;
            s += loc[j];
        }
        long long tot;
        long long ex = run + block_excl_scan<long long>(s, red, tot);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const long long i = i0 + j;
            if (i < W.nseg) W.seg_off[i] = ex;
            ex += loc[j];
        }
        run += tot;
    }
    if (threadIdx.x == 0) W.ctr->punctures = run;
}

// Streaming variants: scan over the segments in face-id order, many blocks
// with decoupled look-back (tiles of SEG_TILE segments).  A segment's count
// is the difference of surv_off across its survivor run, and seg_off[seg] is
// stored minus surv_off at the run's start, so that seg_off[seg] +
// surv_off[s] is the sorted position of survivor s's first puncture.
__global__ void __launch_bounds__(NT) k_seg_scan(Workspace W) {
    constexpr int PER = SEG_TILE / NT;
    __shared__ long long red[NT / 32 + 1];
    __shared__ long long sh[2];
    if (W.ctr->status & ST_SOVERFLOW) return;
    const long long ns = (long long)W.ctr->survivors;
    const long long total = W.ctr->surv_total;
    while (true) {
        if (threadIdx.x == 0) sh[1] = (long long)atomicAdd(&W.ctr->seg_tiles, 1ull);
        __syncthreads();
        const long long t = sh[1];
        if (t * SEG_TILE >= W.nseg) break;
        const long long i0 = t * SEG_TILE + (long long)threadIdx.x * PER;
        // loads are unconditional (clamped indices) so that each round of
        // them is issued at once: the counts, then the offsets they point at
        int n[PER];
        long long a[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const long long i = i0 + j < W.nseg ? i0 + j : 0;
            n[j] = i0 + j < W.nseg ? W.seg_scnt[i] : 0;
            a[j] = W.seg_sstage[i];
        }
        int v1[PER], v2[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const long long e = a[j] + n[j];
            v1[j] = W.surv_off[n[j] > 0 ? a[j] : 0];
            v2[j] = W.surv_off[n[j] > 0 && e < ns ? e : 0];
        }
        long long loc[PER], first[PER];
        long long s = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const long long e = a[j] + n[j];
            first[j] = n[j] > 0 ? v1[j] : 0;
            loc[j] = n[j] > 0 ? (e < ns ? (long long)v2[j] : total) - first[j] : 0;
            s += loc[j];
        }
        long long tot;
        long long ex = block_excl_scan<long long>(s, red, tot);
        if (threadIdx.x < 32) {
            const long long before = warp_lookback(W.seg_tile, t, tot, &W.ctr->status);
            if (threadIdx.x == 0) {
                sh[0] = before;
                if ((t + 1) * SEG_TILE >= W.nseg) {
                    // the last tile: the puncture count; punctures go straight
                    // to their sorted slots
                    const long long run = before + tot;
                    W.ctr->punctures = run;
                    W.ctr->staged = (unsigned long long)run;
                    if (run > W.cap) atomicOr(&W.ctr->status, ST_OVERFLOW);
                }
            }
        }
        __syncthreads();
        ex += sh[0];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            if (i0 + j < W.nseg) W.seg_off[i0 + j] = ex - first[j];
            ex += loc[j];
        }
        __syncthreads();
    }
}


// Hessian entry H_ab = difference of G_a along axis b with the gradient's
// boundary rule.  hess_sym returns every HS_ab = H_ab + H_ba at point p
// (element offset ip) from the distinct samples they use.  Per axis a:
// lo_a = max(p_a - 1, 0), hi_a = min(p_a + 1, n_a - 1), m_a as above, so
// G_a = m_a (f[hi_a] - f[lo_a]) and
//   H_aa = m_a (G_a(p : a -> hi_a) - G_a(p : a -> lo_a)),
//   H_ab = m_a m_b (f[hi_a, hi_b] - f[lo_a, hi_b] - f[hi_a, lo_b] + f[lo_a, lo_b])  (a != b),
// the latter symmetric because a step along b leaves m_a, lo_a, hi_a as
// they are.  With WITH_G, G receives the gradient from the same samples.
template <int N, bool WITH_G = false>
__device__ void hess_sym(const Field &F, const Pt &p, long long ip, long long (&HS)[N][N], int32_t *G = nullptr) {
    long long dlo[N], dhi[N], st[N];
    int m[N], n[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        n[a] = ext_of(F, a);
        st[a] = vstride(F, a);
        dlo[a] = p.c[a] > 0 ? -st[a] : 0;
        dhi[a] = p.c[a] + 1 < n[a] ? st[a] : 0;
        m[a] = (p.c[a] == 0 || p.c[a] == n[a] - 1) ? 2 : 1;
    }
    const int f0 = qat(F, ip);
#pragma unroll
    for (int a = 0; a < N; ++a) {
        const int fh = qat(F, ip + dhi[a]), fl = qat(F, ip + dlo[a]);
        if (WITH_G) G[a] = m[a] * (fh - fl);
        const int hi = p.c[a] + 1 < n[a] ? p.c[a] + 1 : n[a] - 1;
        const int lo = p.c[a] > 0 ? p.c[a] - 1 : 0;
        // G_a at hi_a: samples min(hi_a + 1, n - 1) and max(hi_a - 1, 0)
        const long long h2 = hi + 1 < n[a] ? dhi[a] + st[a] : dhi[a];
        const int gh = (hi == n[a] - 1 ? 2 : 1) * (qat(F, ip + h2) - (hi == p.c[a] ? fl : f0));
        const long long l2 = lo > 0 ? dlo[a] - st[a] : dlo[a];
        const int gl = (lo == 0 ? 2 : 1) * ((lo == p.c[a] ? fh : f0) - qat(F, ip + l2));
        HS[a][a] = 2LL * m[a] * ((long long)gh - gl);
#pragma unroll
        for (int b = a + 1; b < N; ++b) {
            const long long x = (long long)qat(F, ip + dhi[a] + dhi[b]) - qat(F, ip + dlo[a] + dhi[b]) -
                                qat(F, ip + dhi[a] + dlo[b]) + qat(F, ip + dlo[a] + dlo[b]);
            HS[a][b] = HS[b][a] = 2LL * m[a] * m[b] * x;
        }
    }
}


template <int N>
__device__ __forceinline__ Pt decode_face(const Field &F, long long fid, int &tt) {
    constexpr int T = MeshDims<N>::T;
    const long long g = fid / T;
    tt = (int)(fid - g * T);
    return decode_vertex(F, g);
}

// vertex k of a simplex: base + bits of mask m (axis N of m is time)

template <int N, int W>
__device__ int morse_from_S(const BigInt<W> (&S)[N][N]) {
    BigInt<W> e[N];
    if (N == 2) {
        e[0] = big_add(S[0][0], S[1][1]);
        e[1] = big_sub(big_mul(S[0][0], S[1][1]), big_mul(S[0][1], S[1][0]));
    } else {
        e[0] = big_add(big_add(S[0][0], S[1][1]), S[N - 1][N - 1]);
        BigInt<W> m01 = big_sub(big_mul(S[0][0], S[1][1]), big_mul(S[0][1], S[1][0]));
        BigInt<W> m02 = big_sub(big_mul(S[0][0], S[N - 1][N - 1]), big_mul(S[0][N - 1], S[N - 1][0]));
        BigInt<W> m12 = big_sub(big_mul(S[1][1], S[N - 1][N - 1]), big_mul(S[1][N - 1], S[N - 1][1]));
        e[1] = big_add(big_add(m01, m02), m12);
        // det by expansion along row 0
        BigInt<W> c0 = m12;
        BigInt<W> c1 = big_sub(big_mul(S[1][0], S[N - 1][N - 1]), big_mul(S[1][N - 1], S[N - 1][0]));
        BigInt<W> c2 = big_sub(big_mul(S[1][0], S[N - 1][1]), big_mul(S[1][1], S[N - 1][0]));
        e[N - 1] = big_add(big_sub(big_mul(S[0][0], c0), big_mul(S[0][1], c1)), big_mul(S[0][N - 1], c2));
    }
    if (big_sign(e[N - 1]) == 0) return -1;
    int prev = 1, changes = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int s = big_sign(e[i]);
        if (s != 0) {
            if (s != prev) ++changes;
            prev = s;
        }
    }
    return changes;
}

// |a| * |b| as a 256-bit magnitude (hi, lo)
__device__ __forceinline__ void mul_u128(unsigned __int128 a, unsigned __int128 b, unsigned __int128 &hi,
                                         unsigned __int128 &lo) {
    const unsigned long long a0 = (unsigned long long)a, a1 = (unsigned long long)(a >> 64);
    const unsigned long long b0 = (unsigned long long)b, b1 = (unsigned long long)(b >> 64);
    const unsigned __int128 p00 = (unsigned __int128)a0 * b0;
    const unsigned __int128 p01 = (unsigned __int128)a0 * b1;
    const unsigned __int128 p10 = (unsigned __int128)a1 * b0;
    const unsigned __int128 p11 = (unsigned __int128)a1 * b1;
    const unsigned __int128 mid = (p00 >> 64) + (unsigned long long)p01 + (unsigned long long)p10;
    lo = (mid << 64) | (unsigned long long)p00;
    hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
}

// sign(a*b - c*d) for signed 128-bit operands, exact
__device__ int cmp_prod128(__int128 a, __int128 b, __int128 c, __int128 d) {
    const int s1 = sgn128(a) * sgn128(b), s2 = sgn128(c) * sgn128(d);
    if (s1 != s2) return s1 > s2 ? 1 : -1;   // also covers zero products
    if (s1 == 0) return 0;
    unsigned __int128 h1, l1, h2, l2;
    mul_u128(a < 0 ? (unsigned __int128)(-a) : (unsigned __int128)a,
             b < 0 ? (unsigned __int128)(-b) : (unsigned __int128)b, h1, l1);
    mul_u128(c < 0 ? (unsigned __int128)(-c) : (unsigned __int128)c,
             d < 0 ? (unsigned __int128)(-d) : (unsigned __int128)d, h2, l2);
    const int mag = h1 != h2 ? (h1 > h2 ? 1 : -1) : (l1 != l2 ? (l1 > l2 ? 1 : -1) : 0);
    return s1 > 0 ? mag : -mag;   // both products positive, or both negative
}

constexpr int8_t MORSE_PENDING = -2;   // 3D: left to the exact classification

// location and Morse index of one puncture.  In 3D with FILTER_ONLY the
// index comes from the floating-point filter, or MORSE_PENDING when the
// filter cannot certify it (the exact evaluation then runs separately).
// Jacobian of a 2D vector field at p (element offset ip): J_ab = difference
// of component a along axis b with the gradient's rule (central inside,
// one-sided and doubled at either end)
__device__ __forceinline__ void jac_vec2(const Field &F, const Pt &p, long long ip, long long (&J)[2][2]) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int n = ext_of(F, b);
        const long long st = vstride(F, b);
        const long long lo = p.c[b] > 0 ? ip - st : ip;
        const long long hi = p.c[b] + 1 < n ? ip + st : ip;
        const int m = (p.c[b] == 0 || p.c[b] == n - 1) ? 2 : 1;
#pragma unroll
        for (int a = 0; a < 2; ++a) J[a][b] = (long long)m * (qat(F, 2 * hi + a) - qat(F, 2 * lo + a));
    }
}

// Location and type of a zero of a 2D vector field (paper Sec. 4.1: sources,
// sinks and saddles from the Jacobian's eigenvalues).  S = sign(D) sum_k D_k
// J_k, a positive multiple of the interpolated Jacobian (not symmetrised):
// type = number of eigenvalues with negative real part (0 source, 1 saddle,
// 2 sink), -1 when one is zero (det S = 0, or det S > 0 and tr S = 0).
// |V| <= 2^28: D_k < 2^58, |J| < 2^31, entries of S < 2^91 in int128, det S
// compared exactly by cmp_prod128.
__device__ void locate_classify_vec2(const Field &F, long long fid, float4 &off, int8_t &morse) {
    int tt;
    const Pt base = decode_face<2>(F, fid, tt);
    const uint8_t *ch = mesh<2>().face[tt];
    int32_t V[3][2];
    long long J[3][2][2];
    const long long ib = vindex(F, base);
#pragma unroll
    for (int k = 0; k <= 2; ++k) {
        const Pt vk = k == 0 ? base : add_mask<2>(base, ch[k - 1]);
        const long long ik = k == 0 ? ib : ib + mask_offset<2>(F, ch[k - 1]);
        V[k][0] = grad_at(F, vk, ik, 0);
        V[k][1] = grad_at(F, vk, ik, 1);
        jac_vec2(F, vk, ik, J[k]);
    }
    long long D[3], Dsum = 0;
#pragma unroll
    for (int k = 0; k <= 2; ++k) {
        const int j0 = k == 0 ? 1 : 0, j1 = k == 2 ? 1 : 2;
        const long long d = (long long)V[j0][0] * V[j1][1] - (long long)V[j0][1] * V[j1][0];
        D[k] = (k & 1) ? -d : d;
        Dsum += D[k];
    }
    float mu[3];
#pragma unroll
    for (int k = 0; k <= 2; ++k) mu[k] = Dsum == 0 ? 1.0f / 3 : (float)D[k] / (float)Dsum;
    float o[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 1; k <= 2; ++k)
#pragma unroll
        for (int a = 0; a <= 2; ++a)
            if ((ch[k - 1] >> a) & 1) o[a] += mu[k];
    off = make_float4(o[0], o[1], 0.0f, o[2]);
    __int128 S[2][2] = {{0, 0}, {0, 0}};
#pragma unroll
    for (int k = 0; k <= 2; ++k) {
        const __int128 w = Dsum < 0 ? -(__int128)D[k] : (__int128)D[k];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) S[a][b] += w * (__int128)J[k][a][b];
    }
    const int d = cmp_prod128(S[0][0], S[1][1], S[0][1], S[1][0]);   // sign of det S
    const __int128 tr = S[0][0] + S[1][1];
    morse = (int8_t)(d < 0 ? 1 : d == 0 || tr == 0 ? -1 : tr < 0 ? 2 : 0);
}

// 3D location (Eq. 1) and Morse index of a punctured face from its vertices'
// gradients V[k] and symmetrised Hessians HS[k] (k in chain order; ch = the
// face's chain).  FILTER_ONLY: MORSE_PENDING where neither exact int128 nor
// the certified FP32 filter decides (the multiword evaluation is left to a
// later pass).
template <bool FILTER_ONLY>
__device__ void locate_classify3_from(const uint8_t *ch, const int32_t (&V)[4][3], const long long (&HS)[4][3][3],
                                      float4 &off, int8_t &morse) {
    constexpr int N = 3, BW = 16;
    __int128 D[N + 1];
    __int128 Dsum = 0;
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        int32_t M[N][N];
        int c = 0;
#pragma unroll
        for (int j = 0; j <= N; ++j) {
            if (j == k) continue;
#pragma unroll
            for (int r = 0; r < N; ++r) M[c][r] = V[j][r];
            ++c;
        }
        const __int128 d = det_exact(M);
        D[k] = ((N + k) & 1) ? -d : d;
        Dsum += D[k];
    }
    float mu[N + 1];
    if (Dsum == 0) {
#pragma unroll
        for (int k = 0; k <= N; ++k) mu[k] = 1.0f / (N + 1);
    } else {
        const float fd = i128_to_float(Dsum);
#pragma unroll
        for (int k = 0; k <= N; ++k) mu[k] = i128_to_float(D[k]) / fd;
    }
    float o[N + 1];
#pragma unroll
    for (int a = 0; a <= N; ++a) o[a] = 0.0f;
#pragma unroll
    for (int k = 1; k <= N; ++k)
#pragma unroll
        for (int a = 0; a <= N; ++a)
            if ((ch[k - 1] >> a) & 1) o[a] += mu[k];
    off = make_float4(o[0], o[1], o[2], o[N]);

    // S = sign(D) sum_k D_k (H_k + H_k^T), exact
    const int sg = sgn128(Dsum);
    {
        // S exactly in int128 (|w| < 2^93, |h| < 2^34) and in FP32 from
        // weights scaled by one power of two (the index is unchanged by a
        // positive scale).  Small S (every entry < 2^40, e.g. near-flat,
        // quantised regions): tr, m2 and det exactly in int128 (products
        // < 2^121).  Otherwise the FP32 filter, and the multiword evaluation
        // below only when the filter cannot certify every sign.
        __int128 wmax = 0;
        for (int k = 0; k <= N; ++k) {
            const __int128 w = D[k] < 0 ? -D[k] : D[k];
            if (w > wmax) wmax = w;
        }
        const int wbits = i128_bits(wmax);
        __int128 Si[3][3];
        float Sd[3][3], Ad[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                Si[a][b] = 0;
                Sd[a][b] = Ad[a][b] = 0.0f;
            }
        for (int k = 0; k <= N; ++k) {
            const __int128 w = sg < 0 ? -D[k] : D[k];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = a; b < 3; ++b) Si[a][b] += w * (__int128)HS[k][a][b];
            s_fp32_step<3>(ldexpf(i128_to_float(w), 1 - wbits), HS[k], Sd, Ad);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < a; ++b) Si[a][b] = Si[b][a];
        s_fp32_symmetrise<3>(Sd, Ad);
        const __int128 LIM = (__int128)1 << 40;
        // the int128 sums cannot wrap: 4 terms of |w| < 2^wbits, |h| < 2^35
        bool small = wbits <= 88;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) small &= Si[a][b] < LIM && Si[a][b] > -LIM;
        if (small) {
            const __int128 tr = Si[0][0] + Si[1][1] + Si[2][2];
            const __int128 m2 = Si[0][0] * Si[1][1] - Si[0][1] * Si[0][1] + Si[0][0] * Si[2][2] -
                                Si[0][2] * Si[0][2] + Si[1][1] * Si[2][2] - Si[1][2] * Si[1][2];
            const __int128 det = Si[0][0] * (Si[1][1] * Si[2][2] - Si[1][2] * Si[1][2]) -
                                 Si[0][1] * (Si[0][1] * Si[2][2] - Si[1][2] * Si[0][2]) +
                                 Si[0][2] * (Si[0][1] * Si[1][2] - Si[1][1] * Si[0][2]);
            if (det == 0) {
                morse = -1;
                return;
            }
            const int sgn3[3] = {sgn128(tr), sgn128(m2), sgn128(det)};
            int prev = 1, changes = 0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
                if (sgn3[i] != 0) {
                    if (sgn3[i] != prev) ++changes;
                    prev = sgn3[i];
                }
            morse = (int8_t)changes;
            return;
        }
        int m = 0;
        if (morse_filter3(Sd, Ad, m)) {
            morse = (int8_t)m;
            return;
        }
        if constexpr (FILTER_ONLY) {
            morse = MORSE_PENDING;
            return;
        }
    }
    if constexpr (!FILTER_ONLY) {
        BigInt<BW> S[N][N];
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) S[a][b] = big_from<BW>(0);
        for (int k = 0; k <= N; ++k) {
            const __int128 w = sg < 0 ? -D[k] : D[k];
            for (int a = 0; a < N; ++a)
                for (int b = 0; b < N; ++b)
                    S[a][b] = big_add(S[a][b], big_from<BW>(w * (__int128)HS[k][a][b]));
        }
        morse = (int8_t)morse_from_S<N, BW>(S);
    }
}

template <int N, bool FILTER_ONLY = false>
__device__ void locate_classify(const Field &F, long long fid, float4 &off, int8_t &morse) {
    if constexpr (N == 2) {
        if (F.comps == 2) {
            locate_classify_vec2(F, fid, off, morse);
            return;
        }
    }
    int tt;
    const Pt base = decode_face<N>(F, fid, tt);
    const uint8_t *ch = mesh<N>().face[tt];
    Pt v[N + 1];
    long long iv[N + 1];
    int32_t V[N + 1][N];
    long long HS2[N == 2 ? 3 : 1][N][N];   // 2D: every vertex's HS from the same samples as its gradient
    const long long ib = vindex(F, base);
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        v[k] = k == 0 ? base : add_mask<N>(base, ch[k - 1]);
        iv[k] = k == 0 ? ib : ib + mask_offset<N>(F, ch[k - 1]);
        if constexpr (N == 2) hess_sym<N, true>(F, v[k], iv[k], HS2[k], V[k]);
    }
    if constexpr (N == 2) {
        // |G| <= 2^30: the 2x2 determinants (< 2^61) and their sum fit in int64
        long long D[3], Dsum = 0;
#pragma unroll
        for (int k = 0; k <= 2; ++k) {
            const int j0 = k == 0 ? 1 : 0, j1 = k == 2 ? 1 : 2;
            const long long d = (long long)V[j0][0] * V[j1][1] - (long long)V[j0][1] * V[j1][0];
            D[k] = (k & 1) ? -d : d;
            Dsum += D[k];
        }
        float mu[3];
        if (Dsum == 0) {
#pragma unroll
            for (int k = 0; k <= 2; ++k) mu[k] = 1.0f / 3;
        } else {
            const float fd = (float)Dsum;
#pragma unroll
            for (int k = 0; k <= 2; ++k) mu[k] = (float)D[k] / fd;
        }
        float o[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int k = 1; k <= 2; ++k)
#pragma unroll
            for (int a = 0; a <= 2; ++a)
                if ((ch[k - 1] >> a) & 1) o[a] += mu[k];
        off = make_float4(o[0], o[1], 0.0f, o[2]);
        // S = sign(D) sum_k D_k (H_k + H_k^T): FP32 filter, else exact (|w| <
        // 2^62 and |H + H^T| < 2^34: entries in int128, det S compared in 256 bits)
        const bool neg = Dsum < 0;
        long long wmax = 0;
#pragma unroll
        for (int k = 0; k <= 2; ++k) wmax = max(wmax, D[k] < 0 ? -D[k] : D[k]);
        const int wbits = i128_bits(wmax);
        float Sd[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}}, Ad[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll
        for (int k = 0; k <= 2; ++k)
            s_fp32_step<2>(ldexpf(i128_to_float(neg ? -D[k] : D[k]), 1 - wbits), HS2[k], Sd, Ad);
        s_fp32_symmetrise<2>(Sd, Ad);
        int m = 0;
        if (morse_filter2(Sd, Ad, m)) {
            morse = (int8_t)m;
            return;
        }
        __int128 S00 = 0, S01 = 0, S11 = 0;
#pragma unroll
        for (int k = 0; k <= 2; ++k) {
            const __int128 w = neg ? -(__int128)D[k] : (__int128)D[k];
            S00 += w * (__int128)HS2[k][0][0];
            S11 += w * (__int128)HS2[k][1][1];
            S01 += w * (__int128)HS2[k][0][1];
        }
        const int d = cmp_prod128(S00, S11, S01, S01);   // sign(S00 S11 - S01 S01)
        const __int128 tr = S00 + S11;
        morse = (int8_t)(d < 0 ? 1 : d > 0 ? (tr < 0 ? 2 : 0) : -1);
        return;
    } else {
        long long HS3[4][3][3];
#pragma unroll
        for (int k = 0; k <= 3; ++k) hess_sym<3, true>(F, v[k], iv[k], HS3[k], V[k]);
        locate_classify3_from<FILTER_ONLY>(ch, V, HS3, off, morse);
    }   // N == 3
}

template <int N>
__global__ void __launch_bounds__(NT) k_finalize(Field F, Blocking B, Workspace W) {
    const unsigned long long staged_all = W.ctr->staged;
    const long long staged = staged_all < (unsigned long long)W.cap ? (long long)staged_all : W.cap;
    if (W.ctr->status & ST_OVERFLOW) return;
    constexpr int T = MeshDims<N>::T;
    for (long long s = blockIdx.x * (long long)NT + threadIdx.x; s < staged; s += (long long)gridDim.x * NT) {
        const long long fid = W.staging[s];
        const long long seg = segment_of(fid / T, F, B);
        const long long i = W.seg_off[seg] + (s - W.seg_stage[seg]);
        W.face[i] = fid;
        W.parent[i] = (int)i;
        float4 o;
        int8_t m;
        locate_classify<N>(F, fid, o, m);
        W.off[i] = o;
        W.morse[i] = m;
    }
}

// ----------------------------------------------------------------------------
// Linking
// ----------------------------------------------------------------------------
__device__ __forceinline__ int uf_find(int *parent, int x, unsigned *status, int lim = UF_LIMIT) {
    for (int it = 0; it < lim; ++it) {
        const int p = *(volatile int *)&parent[x];
        if (p == x) return x;
        const int gp = *(volatile int *)&parent[p];
        if (gp != p) *(volatile int *)&parent[x] = gp;   // path halving (points to an ancestor)
        x = gp;
    }
    atomicOr(status, ST_TIMEOUT);
    return x;
}

__device__ __forceinline__ void uf_unite(int *parent, int a, int b, unsigned *status, int lim = UF_LIMIT) {
    for (int it = 0; it < lim; ++it) {
        a = uf_find(parent, a, status, lim);
        b = uf_find(parent, b, status, lim);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        // hook the larger root under the smaller: roots stay component minima
        const int old = atomicCAS(&parent[a], a, b);
        if (old == a) return;
        a = old;
    }
    atomicOr(status, ST_TIMEOUT);
}

template <int N>
__device__ __forceinline__ long long face_id_of(const Field &F, Pt b, const int (&m)[N]) {
    constexpr int T = MeshDims<N>::T;
    const int tt = mesh<N>().lookup[chain_key<N>(m)];
    const long long g = (((long long)b.c[3] * F.nz + b.c[2]) * F.ny + b.c[1]) * F.nx + b.c[0];
    return g * T + tt;
}

// index of face `key` (base vertex b) in the sorted array, searching only
// its own segment
__device__ __forceinline__ long long find_in_segment(const Field &F, const Blocking &B, const Workspace &W,
                                                     const Pt &b, long long key) {
    const long long seg = segment_of_coords(b.c[0], b.c[1], b.c[2], b.c[3], F, B);
    const long long lo0 = W.seg_off[seg];
    const long long hi0 = lo0 + W.seg_cnt[seg];
    long long lo = lo0, hi = hi0;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (W.face[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < hi0 && W.face[lo] == key) ? lo : -1;
}

template <int N>
__global__ void __launch_bounds__(NT) k_link(Field F, Blocking B, Workspace W) {
    constexpr int D = N + 1;
    constexpr int FULL = (1 << D) - 1;
    if (W.ctr->status & (ST_OVERFLOW | ST_SOVERFLOW)) return;
    const long long P = W.ctr->punctures;
    unsigned *status = &W.ctr->status;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < P; i += (long long)gridDim.x * NT) {
        const long long fid = W.face[i];
        int tt;
        const Pt base = decode_face<N>(F, fid, tt);
        int m[N];
        for (int k = 0; k < N; ++k) m[k] = mesh<N>().face[tt][k];
        // cofaces: cells (base, full chain of D masks) containing the face
        Pt cb[2];
        int cm[2][D];
        int ncell = 0;
        if (m[N - 1] == FULL) {
            int prev = 0;
            for (int j = 0; j < N; ++j) {
                const int step = m[j] ^ prev;
                if (__popc(step) == 2) {
                    for (int a = 0; a < D; ++a) {
                        if (!((step >> a) & 1)) continue;
                        for (int q = 0; q < j; ++q) cm[ncell][q] = m[q];
                        cm[ncell][j] = prev | (1 << a);
                        for (int q = j; q < N; ++q) cm[ncell][q + 1] = m[q];
                        cb[ncell] = base;
                        ++ncell;
                    }
                    break;
                }
                prev = m[j];
            }
        } else {
            const int a = __ffs(FULL ^ m[N - 1]) - 1;
            const int ca = a == N ? 3 : a;           // coordinate slot of axis a
            const int ext = a == N ? F.nt : (a == 0 ? F.nx : a == 1 ? F.ny : F.nz);
            if (base.c[ca] >= 1) {
                cb[ncell] = base;
                cb[ncell].c[ca] -= 1;
                cm[ncell][0] = 1 << a;
                for (int q = 0; q < N; ++q) cm[ncell][q + 1] = m[q] | (1 << a);
                ++ncell;
            }
            if (base.c[ca] + 1 < ext) {
                cb[ncell] = base;
                for (int q = 0; q < N; ++q) cm[ncell][q] = m[q];
                cm[ncell][N] = FULL;
                ++ncell;
            }
        }
        for (int c = 0; c < ncell; ++c) {
            int hits = 0;
            long long partner = -1;
            for (int k = 0; k <= D; ++k) {
                Pt sb = cb[c];
                int sm[N];
                if (k == 0) {
                    sb = add_mask<N>(cb[c], cm[c][0]);
                    for (int q = 0; q < N; ++q) sm[q] = cm[c][q + 1] ^ cm[c][0];
                } else if (k == D) {
                    for (int q = 0; q < N; ++q) sm[q] = cm[c][q];
                } else {
                    int w = 0;
                    for (int q = 0; q < D; ++q)
                        if (q != k - 1) sm[w++] = cm[c][q];
                }
                const long long sid = face_id_of<N>(F, sb, sm);
                if (sid == fid) continue;
                const long long j = find_in_segment(F, B, W, sb, sid);
                if (j >= 0) { ++hits; partner = j; }
            }
            if (hits != 1) {
                atomicOr(status, ST_PAIRING);
                continue;
            }
            // both ends see the pair; one union suffices
            if (partner > i) uf_unite(W.parent, (int)i, (int)partner, status);
        }
    }
}

// survivor index of the cube based at vertex b (its segment's survivors are
// sorted by vertex id), or -1 if the cube did not survive the cull (then
// none of its faces is punctured)
__device__ __forceinline__ long long find_cube(const Field &F, const Blocking &B, const Workspace &W, const Pt &b) {
    const long long seg = segment_of_coords(b.c[0], b.c[1], b.c[2], b.c[3], F, B);
    const long long lo0 = W.seg_sstage[seg];
    const long long hi0 = lo0 + W.seg_scnt[seg];
    const long long key = (((long long)b.c[3] * F.nz + b.c[2]) * F.ny + b.c[1]) * F.nx + b.c[0];
    long long lo = lo0, hi = hi0;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (W.surv[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < hi0 && W.surv[lo] == key) ? lo : -1;
}

// number of cells having face type tt based at b as a side
template <int N>
__device__ __forceinline__ int face_cells(const Field &F, const Pt &b, int tt) {
    constexpr int FULL = MeshDims<N>::FULL;
    const int last = mesh<N>().face[tt][N - 1];
    if (last == FULL) return 2;                      // inside the cube: both cells in it
    const int a = __ffs(FULL ^ last) - 1;            // the face lies in the plane x_a = b_a
    // selects, not a runtime index into b (which would move b to local memory)
    const int x = a == 0 ? b.c[0] : a == 1 ? b.c[1] : a == N ? b.c[3] : b.c[2];
    const int ext = a == N ? F.nt : ext_of(F, a);
    return (x >= 1) + (x + 1 < ext);
}

// Linking for the streaming variants (Algorithm 1, second loop), one thread
// per surviving cube: every cell lies in exactly one unit cube, and a cell
// with a punctured side has one through the cube's base vertex (its sides
// through b are faces of the cube at b; the opposite side belongs to the next
// cube along the cell's first step, found in the survivor list).  A cell
// with exactly two punctured sides joins them; one with any other nonzero
// count breaks the pairing invariant.  Cells whose sides through b are all
// unpunctured are not visited: each of them must then have no punctured side
// at all, which the global count checks -- every punctured face lies in one
// or two cells (one on the grid boundary), so the cells visited with two
// punctured sides must number exactly half the sum of those counts.
template <int N>
__global__ void __launch_bounds__(NT, 6) k_link_survivors(Field F, Blocking B, Workspace W) {
    constexpr int D = N + 1;
    constexpr int FULL = (1 << D) - 1;
    constexpr int C = MeshDims<N>::C;
    __shared__ unsigned long long red[2][NT / 32];
    if (W.ctr->status & (ST_OVERFLOW | ST_SOVERFLOW)) return;
    const long long P = W.ctr->punctures;
    unsigned *status = &W.ctr->status;
    unsigned long long pairs = 0, incid = 0;
    // one item per (surviving cube, first-step axis a): the cells of the cube
    // that step first along a, all of which share the next cube along a.
    // Items are axis-major, so a warp's lanes take the same branch (a search
    // for the next cube along y, z or t; none along x).
    // 2D: the items come from the lists the survivor evaluation filled, taken
    // one after the other (every lane of a warp holds a real item; each list
    // holds fewer than scap <= 2^26 items).  3D (few survivors): every
    // (survivor, axis) pair, axis-major, filtered here.
    const long long ns = (long long)W.ctr->survivors;
    int bnd[D];                  // 2D: bnd[a] = items in the lists up to a
    {
        int run = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            run += N == 2 ? (int)W.ctr->nlink[a] : 0;
            bnd[a] = run;
        }
    }
    const long long total = N == 2 ? (long long)bnd[D - 1] : ns * D;
    for (long long it = blockIdx.x * (long long)NT + threadIdx.x; it < total; it += (long long)gridDim.x * NT) {
        int a = 0;
        long long s;
        if constexpr (N == 2) {
#pragma unroll
            for (int q = 0; q + 1 < D; ++q) a += it >= bnd[q];
            const int k = (int)it - (a == 0 ? 0 : a == 1 ? bnd[0] : bnd[1]);
            s = W.litem[(long long)a * W.scap + k];
        } else {
            a = (int)(it / ns);
            s = it - (long long)a * ns;
        }
        const unsigned long long mo = W.surv_mask[s];
        if (!mo || (a != 0 && !(mo & cells<N>().own_axis[a]))) continue;
        const long long g = W.surv[s];
        const Pt b = decode_vertex(F, g);
        if (a == 0) {   // the item of axis 0 also counts the cube's face incidences
            for (unsigned long long r = mo; r; r &= r - 1) incid += face_cells<N>(F, b, __ffsll((long long)r) - 1);
            if (!(mo & cells<N>().own_axis[0])) continue;
        }
        int inside = 0;
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const int slot = q == N ? 3 : q;
            const int ext = q == N ? F.nt : ext_of(F, q);
            if (b.c[slot] + 1 < ext) inside |= 1 << q;
        }
        if (inside != FULL) continue;                // a boundary cube holds no cell
        const long long seg = segment_of_coords(b.c[0], b.c[1], b.c[2], b.c[3], F, B);
        const long long pos = W.seg_off[seg] + W.surv_off[s];
        // the next cube along axis a: its mask and first puncture's position
        unsigned long long mf = 0;
        long long pf = 0;
        if (a == 0) {
            // the next vertex id: the next survivor of the segment, if any
            const long long e = W.seg_sstage[seg] + W.seg_scnt[seg];
            if (s + 1 < e && W.surv[s + 1] == g + 1) {
                mf = W.surv_mask[s + 1];
                pf = pos + __popcll(mo);
            }
        } else {
            Pt q = b;   // b + e_a, without a runtime index into q
            q.c[1] += a == 1;
            q.c[2] += N == 3 && a == 2;
            q.c[3] += a == N;
            const long long sf = find_cube(F, B, W, q);
            if (sf >= 0) {
                mf = W.surv_mask[sf];
                pf = W.seg_off[segment_of_coords(q.c[0], q.c[1], q.c[2], q.c[3], F, B)] + W.surv_off[sf];
            }
        }
        constexpr int PER = C / D;
        for (int c = a * PER; c < (a + 1) * PER; ++c) {
            const unsigned long long in_own = mo & cells<N>().own[c];
            if (!in_own) continue;
            const int ft = cells<N>().far[c];
            const bool far_hit = (mf >> ft) & 1ull;
            const int n = __popcll(in_own) + (far_hit ? 1 : 0);
            if (n != 2) {
                atomicOr(status, ST_PAIRING);
                continue;
            }
            const int t0 = __ffsll((long long)in_own) - 1;
            const long long i = pos + __popcll(mo & ((1ull << t0) - 1ull));
            long long j;
            if (far_hit) {
                j = pf + __popcll(mf & ((1ull << ft) - 1ull));
            } else {
                const int t1 = __ffsll((long long)(in_own & (in_own - 1))) - 1;
                j = pos + __popcll(mo & ((1ull << t1) - 1ull));
            }
            if (i < 0 || j < 0 || i >= P || j >= P) {   // only after a failed scan (flagged)
                atomicOr(status, ST_PAIRING);
                continue;
            }
            uf_unite(W.parent, (int)i, (int)j, status);
            ++pairs;
        }
    }
    // block totals of the two counts, then one atomic each
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        incid += __shfl_xor_sync(0xffffffffu, incid, o);
    }
    if (lane == 0) { red[0][warp] = pairs; red[1][warp] = incid; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long p = 0, q = 0;
        for (int w = 0; w < NT / 32; ++w) { p += red[0][w]; q += red[1][w]; }
        if (p) atomicAdd(&W.ctr->pairs, p);
        if (q) atomicAdd(&W.ctr->incid, q);
    }
}

template <int N, bool LIM>
__global__ void __launch_bounds__(NT) k_label(Field F, Workspace W, int check_cells) {
    // a block's records are built in shared memory and stored as one
    // contiguous run of 16-byte words (a record is 56 bytes; a run starts at
    // a multiple of NT records, so at a 16-byte boundary)
    static_assert(sizeof(ftk_cp) == 56 && (NT * sizeof(ftk_cp)) % 16 == 0, "record layout");
    __shared__ __align__(16) ftk_cp recs[NT];
    if (W.ctr->status & (ST_OVERFLOW | ST_SOVERFLOW)) return;
    const long long P = W.ctr->punctures;
    unsigned *status = &W.ctr->status;
    // every punctured side of a cell linked exactly once (see k_link_survivors)
    if (check_cells && blockIdx.x == 0 && threadIdx.x == 0 && 2 * W.ctr->pairs != W.ctr->incid)
        atomicOr(status, ST_PAIRING);
    for (long long i0 = blockIdx.x * (long long)NT; i0 < P; i0 += (long long)gridDim.x * NT) {
        const long long i = i0 + threadIdx.x;
        if (i < P) {
            // the run-time bound only in the instance a test selects (a
            // compile-time bound keeps the loop of the normal instance lean)
            const int r = uf_find(W.parent, (int)i, status, LIM ? W.uf_limit : UF_LIMIT);
            const long long fid = W.face[i];
            const long long lab = W.face[r];
            W.label[i] = lab;
            int tt;
            const Pt b = decode_face<N>(F, fid, tt);
            ftk_cp &rec = recs[threadIdx.x];
            rec.face_id = fid;
            rec.label = lab;
            rec.base[0] = b.c[0]; rec.base[1] = b.c[1]; rec.base[2] = b.c[2]; rec.base[3] = b.c[3];
            const float4 o = W.off[i];
            rec.off[0] = o.x; rec.off[1] = o.y; rec.off[2] = o.z; rec.off[3] = o.w;
            rec.morse_index = W.morse[i];
            rec.ordinal = (mesh<N>().face[tt][N - 1] & MeshDims<N>::TBIT) ? 0 : 1;
            rec.ndim = (uint8_t)N;
            for (int q = 0; q < 5; ++q) rec.reserved[q] = 0;
        }
        __syncthreads();
        const long long n = P - i0 < NT ? P - i0 : NT;
        const int nbytes = (int)n * (int)sizeof(ftk_cp);
        const uint4 *src = reinterpret_cast<const uint4 *>(recs);
        uint4 *dst = reinterpret_cast<uint4 *>(W.packed + i0);
        for (int k = threadIdx.x; k < nbytes / 16; k += NT) dst[k] = src[k];
        if ((nbytes & 15) && threadIdx.x == 0) {   // odd count: the last 8 bytes
            const int k = nbytes / 8 - 1;
            reinterpret_cast<unsigned long long *>(W.packed + i0)[k] = reinterpret_cast<const unsigned long long *>(recs)[k];
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// Surviving cubes of the streaming variant: exact evaluation, ordered output
// ----------------------------------------------------------------------------
// bit tt of the result set iff face type tt based at vertex g is punctured
// mask k of the chain of 2D face type tt, evaluated at compile time
__host__ __device__ constexpr int face2_mask(int tt, int k) { return MeshTables<2>().face[tt][k]; }

// the 12 face types of a 2D cube, unrolled at compile time
template <int TT>
__device__ __forceinline__ void eval_faces2(const int32_t (&Gc)[8][2], int inside, unsigned long long &m) {
    if constexpr (TT < MeshDims<2>::T) {
        constexpr int c1 = face2_mask(TT, 0), c2 = face2_mask(TT, 1);
        if (!(c2 & ~inside)) {   // else the face leaves the grid
            const int32_t V[3][2] = {{Gc[0][0], Gc[0][1]}, {Gc[c1][0], Gc[c1][1]}, {Gc[c2][0], Gc[c2][1]}};
            if (face_punctured<2>(V)) m |= 1ull << TT;
        }
        eval_faces2<TT + 1>(Gc, inside, m);
    }
}

// 2D: the link items of surviving cube s with punctured-type mask m: one per
// first-step axis a whose cells the cube owns (axis 0 whenever m != 0: its
// item also counts the cube's face incidences), appended to list a, one
// atomic per warp and list.  The lists' order does not matter: the unions
// they drive end in the same partition, labelled by its smallest face ids.
template <int N>
__device__ __forceinline__ void push_link_items(const Workspace &W, long long s, unsigned long long m) {
    static_assert(N == 2, "the link item lists serve the 2D pipeline");
    constexpr int D = N + 1;
    const unsigned am = __activemask();
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const bool want = m != 0 && (a == 0 || (m & cells<N>().own_axis[a]) != 0);
        const unsigned b = __ballot_sync(am, want);
        if (!b) continue;
        const int lead = __ffs(b) - 1;
        unsigned long long base = 0;
        if (lane == lead) base = atomicAdd(&W.ctr->nlink[a], (unsigned long long)__popc(b));
        base = __shfl_sync(am, base, lead);
        if (want) W.litem[(long long)a * W.scap + (long long)base + __popc(b & ((1u << lane) - 1u))] = (int)s;
    }
}

template <int N>
__device__ unsigned long long eval_cube(const Field &F, long long g) {
    constexpr int D = N + 1;
    constexpr int NCRN = 1 << D;
    constexpr int T = MeshDims<N>::T;
    const Pt b = decode_vertex(F, g);
    int inside = 0;   // bit a: axis a can step +1
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int slot = a == N ? 3 : a;
        const int ext = a == N ? F.nt : ext_of(F, a);
        if (b.c[slot] + 1 < ext) inside |= 1 << a;
    }
    int32_t Gc[NCRN][N];
    const long long ib = vindex(F, b);
#pragma unroll
    for (int c = 0; c < NCRN; ++c) {
        if (c & ~inside) {
#pragma unroll
            for (int r = 0; r < N; ++r) Gc[c][r] = 0;
            continue;
        }
        const Pt p = add_mask<N>(b, c);
        const long long ip = ib + mask_offset<N>(F, c);
#pragma unroll
        for (int r = 0; r < N; ++r) Gc[c][r] = grad_at(F, p, ip, r);
    }
    unsigned long long m = 0;
    if constexpr (N == 2) {
        // face chains as compile-time constants: Gc stays in registers
        eval_faces2<0>(Gc, inside, m);
    } else {
        for (int tt = 0; tt < T; ++tt) {
            const uint8_t *ch = mesh<N>().face[tt];
            if (ch[N - 1] & ~inside) continue;   // the face leaves the grid
            int32_t V[N + 1][N];
#pragma unroll
            for (int k = 0; k <= N; ++k) {
                const int c = k == 0 ? 0 : ch[k - 1];
#pragma unroll
                for (int r = 0; r < N; ++r) V[k][r] = Gc[c][r];
            }
            if (face_punctured<N>(V)) m |= 1ull << tt;
        }
    }
    return m;
}

// The look-back states of this run's two scans start at zero: cleared here,
// by the kernel that precedes both scans, so that no run depends on an
// earlier one having finished (or having run at all).
__device__ __forceinline__ void clear_scan_states(const Workspace &W) {
    const long long ns = (long long)W.ctr->survivors;
    const long long nst = ((ns < W.scap ? ns : W.scap) + LB_TILE - 1) / LB_TILE;
    const long long nsg = (W.nseg + SEG_TILE - 1) / SEG_TILE;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nst + nsg; t += stride) {
        if (t < nst) W.tile[t] = 0ull;
        else W.seg_tile[t - nst] = 0ull;
    }
}

// one thread per surviving cube (grid-stride over the survivor list): the
// form for 2D, whose cubes have few corners and faces
template <int N>
__global__ void __launch_bounds__(NT) k_survive_eval_thread(Field F, Workspace W) {
    clear_scan_states(W);
    if (W.ctr->status & ST_SOVERFLOW) return;
    const long long ns = (long long)W.ctr->survivors;
    for (long long s = blockIdx.x * (long long)NT + threadIdx.x; s < ns; s += (long long)gridDim.x * NT) {
        const unsigned long long m = eval_cube<N>(F, W.surv[s]);
        W.surv_mask[s] = m;
        push_link_items<N>(W, s, m);
    }
}

// 3D: two surviving cubes per warp per step (grid-stride over pairs of the
// survivor list), evaluated by eval_pair3; this kernel also clears the
// look-back states of the run's scans, which follow it
__global__ void __launch_bounds__(NT) k_survive_eval3(Field F, Workspace W) {
    constexpr int WPB = NT / 32;
    __shared__ int32_t Gs[WPB][2][16][3];
    __shared__ uint32_t fch[MeshDims<3>::T];   // face chains m_1 | m_2 << 8 | m_3 << 16
    for (int i = threadIdx.x; i < MeshDims<3>::T; i += NT)
        fch[i] = mesh<3>().face[i][0] | (uint32_t)mesh<3>().face[i][1] << 8 | (uint32_t)mesh<3>().face[i][2] << 16;
    __syncthreads();
    clear_scan_states(W);
    if (W.ctr->status & ST_SOVERFLOW) return;
    const long long ns = (long long)W.ctr->survivors;
    const int warp = threadIdx.x >> 5;
    const Pair3Lane L = pair3_lane(fch);
    const long long stride = (long long)gridDim.x * WPB * 2;
    for (long long s0 = ((long long)blockIdx.x * WPB + warp) * 2; s0 < ns; s0 += stride)
        eval_pair3(F, W, s0, ns, Gs[warp], fch, L);
}

// Offsets of the punctured faces over the survivor list: surv_off[s] = number
// of punctures of the survivors before s in list order (every segment's
// survivors are one contiguous run of the list, so differences give the
// within-segment offsets and the segment totals).  Blocks claim tiles of
// LB_TILE survivors in order; a thread sums the popcounts of LB_TILE / NT
// consecutive masks.
__global__ void __launch_bounds__(NT) k_survive_scan(Workspace W) {
    constexpr int PER = LB_TILE / NT;
    __shared__ long long red[NT / 32 + 1];
    __shared__ long long sh[2];
    if (W.ctr->status & ST_SOVERFLOW) return;
    const long long ns = (long long)W.ctr->survivors;
    while (true) {
        if (threadIdx.x == 0) sh[1] = (long long)atomicAdd(&W.ctr->tiles, 1ull);
        __syncthreads();
        const long long t = sh[1];
        if (t * LB_TILE >= ns) break;
        const long long s0 = t * LB_TILE + (long long)threadIdx.x * PER;
        int c[PER];
        int loc = 0;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            c[k] = s0 + k < ns ? __popcll(W.surv_mask[s0 + k]) : 0;
            loc += c[k];
        }
        long long tot;
        long long ex = block_excl_scan<long long>(loc, red, tot);
        if (threadIdx.x < 32) {
            const long long before = warp_lookback(W.tile, t, tot, &W.ctr->status);
            if (threadIdx.x == 0) {
                sh[0] = before;
                if ((t + 1) * LB_TILE >= ns) W.ctr->surv_total = before + tot;
            }
        }
        __syncthreads();
        ex += sh[0];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (s0 + k < ns) W.surv_off[s0 + k] = (int)(ex < INT_MAX ? ex : INT_MAX);
            ex += c[k];
        }
        __syncthreads();
    }
}

// per surviving cube: write its punctured faces at their sorted positions
template <int N>
__global__ void __launch_bounds__(NT) k_emit(Field F, Blocking B, Workspace W) {
    constexpr int T = MeshDims<N>::T;
    if (W.ctr->status & (ST_OVERFLOW | ST_SOVERFLOW)) return;
    const unsigned long long ns = W.ctr->survivors;
    const long long P = W.ctr->punctures;
    for (long long s = blockIdx.x * (long long)NT + threadIdx.x; s < (long long)ns; s += (long long)gridDim.x * NT) {
        unsigned long long m = W.surv_mask[s];
        if (!m) continue;
        const long long g = W.surv[s];
        long long i = W.seg_off[segment_of(g, F, B)] + W.surv_off[s];
        if (i < 0 || i + __popcll(m) > P) {   // only after a failed scan (flagged)
            atomicOr(&W.ctr->status, ST_PAIRING);
            continue;
        }
        while (m) {
            const int tt = __ffsll((long long)m) - 1;
            m &= m - 1;
            W.face[i] = g * T + tt;
            W.parent[i] = (int)i;
            ++i;
        }
    }
}

// per puncture: location and Morse type
template <int N>
__global__ void __launch_bounds__(NT) k_locate(Field F, Workspace W) {
    if (W.ctr->status & (ST_OVERFLOW | ST_SOVERFLOW)) return;
    const long long P = W.ctr->punctures;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        float4 o;
        int8_t mo;
        locate_classify<N, N == 3>(F, W.face[i], o, mo);
        W.off[i] = o;
        W.morse[i] = mo;
        if (N == 3 && mo == MORSE_PENDING) {
            // W.label is free until k_label: the list of pending punctures
            const unsigned long long q = atomicAdd(&W.ctr->pending, 1ull);
            W.label[q] = i;
        }
    }
}

// 3D, four lanes per puncture: lane k of a group loads vertex k's samples
// (gradient and symmetrised Hessian, all loads issued together), the
// group's first lane locates and classifies the face from them
__global__ void __launch_bounds__(NT) k_locate3(Field F, Workspace W) {
    __shared__ int32_t Vs[NT][3];
    __shared__ long long Hs[NT][6];   // HS_00, 01, 02, 11, 12, 22
    if (W.ctr->status & (ST_OVERFLOW | ST_SOVERFLOW)) return;
    const long long P = W.ctr->punctures;
    const int k = threadIdx.x & 3, g0 = threadIdx.x & ~3;
    for (long long i0 = (long long)blockIdx.x * (NT / 4); i0 < P; i0 += (long long)gridDim.x * (NT / 4)) {
        const long long i = i0 + (threadIdx.x >> 2);
        const bool have = i < P;
        int tt = 0;
        if (have) {
            const Pt base = decode_face<3>(F, W.face[i], tt);
            const int m = k == 0 ? 0 : mesh<3>().face[tt][k - 1];
            const Pt v = add_mask<3>(base, m);
            long long HS[3][3];
            int32_t G[3];
            hess_sym<3, true>(F, v, vindex(F, base) + mask_offset<3>(F, m), HS, G);
            Vs[threadIdx.x][0] = G[0]; Vs[threadIdx.x][1] = G[1]; Vs[threadIdx.x][2] = G[2];
            Hs[threadIdx.x][0] = HS[0][0]; Hs[threadIdx.x][1] = HS[0][1]; Hs[threadIdx.x][2] = HS[0][2];
            Hs[threadIdx.x][3] = HS[1][1]; Hs[threadIdx.x][4] = HS[1][2]; Hs[threadIdx.x][5] = HS[2][2];
        }
        __syncwarp();
        if (have && k == 0) {
            int32_t V[4][3];
            long long HS[4][3][3];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int r = 0; r < 3; ++r) V[q][r] = Vs[g0 + q][r];
                const long long *h = Hs[g0 + q];
                HS[q][0][0] = h[0]; HS[q][0][1] = HS[q][1][0] = h[1]; HS[q][0][2] = HS[q][2][0] = h[2];
                HS[q][1][1] = h[3]; HS[q][1][2] = HS[q][2][1] = h[4]; HS[q][2][2] = h[5];
            }
            float4 o;
            int8_t mo;
            locate_classify3_from<true>(mesh<3>().face[tt], V, HS, o, mo);
            W.off[i] = o;
            W.morse[i] = mo;
            if (mo == MORSE_PENDING) {
                // W.label is free until k_label: the list of pending punctures
                const unsigned long long q = atomicAdd(&W.ctr->pending, 1ull);
                W.label[q] = i;
            }
        }
        __syncwarp();
    }
}

// 3D: exact (multiword) Morse index of the punctures the filter left
template <int N>
__global__ void __launch_bounds__(NT) k_classify_exact(Field F, Workspace W) {
    if (W.ctr->status & (ST_OVERFLOW | ST_SOVERFLOW)) return;
    const long long n = (long long)W.ctr->pending;
    for (long long q = blockIdx.x * (long long)NT + threadIdx.x; q < n; q += (long long)gridDim.x * NT) {
        const long long i = W.label[q];
        float4 o;
        int8_t mo;
        locate_classify<N, false>(F, W.face[i], o, mo);
        W.morse[i] = mo;
    }
}

// ----------------------------------------------------------------------------
// Host-side launch helpers
// ----------------------------------------------------------------------------
cudaError_t raise_smem_cap(const void *kernel, size_t smem, bool capturing) {
    static std::mutex mu;
    static const void *keys[32];
    static size_t caps[32];
    static int n = 0;
    std::lock_guard<std::mutex> lock(mu);
    int i = 0;
    while (i < n && keys[i] != kernel) ++i;
    if (i == n) {
        if (n == 32) return cudaErrorInvalidValue;   // more kernels than the library has
        keys[n] = kernel;
        caps[n] = 0;
        ++n;
    }
    if (smem <= caps[i]) return cudaSuccess;
    if (capturing) return cudaErrorInvalidValue;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) caps[i] = smem;
    return e;
}

size_t detect_smem_bytes(int ndim, const Field &F, const Blocking &B) {
    const int wx = B.nxb > 1 ? B.wx : F.nx;
    const DetectLayout L = ndim == 2 ? detect_layout<2>(wx, B.ry, B.rz, F.comps) : detect_layout<3>(wx, B.ry, B.rz);
    return (size_t)L.total;
}

// four blocks per SM (initialised once, thread-safe)
static int sparse_grid() {
    static const int g = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return (sms > 0 ? sms : 148) * 4;
    }();
    return g;
}

// grid of a latency-bound grid-stride kernel: every block it can keep
// resident on every SM (more loads in flight than sparse_grid's 4 per SM)
template <auto K>
static int resident_grid() {
    static const int g = [] {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K, NT, 0) != cudaSuccess || per < 1) {
            cudaGetLastError();
            per = 4;
        }
        return (sms > 0 ? sms : 148) * per;
    }();
    return g;
}

// ----------------------------------------------------------------------------
// In-situ streaming: merging one push (a 2-slice or 1-slice run) into the
// stream's global union-find over every puncture seen so far.
//
// Push k runs the pipeline on slices [k-1, k] (k = 0: slice 0 alone).  The
// run's punctures get global slots gi = n + i.  Ordinal faces of the run's
// first slice were already reported by push k-1: they are "shadows", linked
// to their earlier slot through push k-1's sorted list of last-slice ordinal
// faces.  Component minima (face ids) are kept at union-find roots; a delta
// label is the minimum over every face known so far that is connected to the
// face.  The stream's scalars (n, k, ordinal counts) live on the device and
// the last merge kernel advances them, so the whole push can be a replayed
// graph.  A run whose pipeline status is bad (range, overflow, exact re-run
// needed) is not merged: the host repairs the run and merges it again.
// ----------------------------------------------------------------------------
constexpr unsigned RUN_BAD = ST_RANGE | ST_OVERFLOW | ST_SOVERFLOW | ST_WIDE | ST_TIMEOUT | ST_PAIRING;

__device__ __forceinline__ bool run_is_shadow(const StreamMerge &M, long long k, long long fid_local) {
    if (k == 0) return false;
    const long long g = fid_local / M.T;
    const int tt = (int)(fid_local - g * M.T);
    return g < M.slice_verts && !(M.tbit & (M.T == 12 ? mesh<2>().face[tt][1] : mesh<3>().face[tt][2]));
}

// slot of a face in a sorted array (or -1)
__device__ __forceinline__ long long bsearch_ll(const long long *a, long long n, long long key) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && a[lo] == key) ? lo : -1;
}

__global__ void __launch_bounds__(NT) k_stream_place(const StreamMerge *__restrict__ Mp) {
    const StreamMerge &M = *Mp;
    if (M.ctr->status & RUN_BAD) return;
    const long long P = M.ctr->punctures;
    const long long k = M.S->k, n_base = M.S->n;
    const int pp = (int)((k - 1) & 1);
    const long long shift_t = k == 0 ? 0 : k - 1;
    const long long shift_g = shift_t * M.slice_verts;
    const long long n_ord = k == 0 ? 0 : M.S->n_ord[pp];
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < P; i += (long long)gridDim.x * NT) {
        const long long gi = n_base + i;
        const long long fl = M.face[i];
        const long long fg = fl + shift_g * M.T;
        const bool sh = run_is_shadow(M, k, fl);
        M.gfid[gi] = fg;
        M.gparent[gi] = (int)gi;
        M.gmin[gi] = sh ? LLONG_MAX : fg;
        M.gshadow[gi] = sh ? 1 : 0;
        ftk_cp r = M.packed[i];
        r.face_id = fg;
        r.base[3] += (int32_t)shift_t;
        M.grec[gi] = r;
        int lp = -1, orr = -1;
        if (sh) {
            const long long j = bsearch_ll(M.ord_fid[pp], n_ord, fg);
            if (j < 0) atomicOr(&M.S->status, ST_PAIRING);   // must have been reported before
            else {
                lp = M.ord_gi[pp][j];
                orr = uf_find(M.gparent, lp, &M.S->status);
            }
        }
        M.link_prev[i] = lp;
        M.old_root[i] = orr;
    }
}

__global__ void __launch_bounds__(NT) k_stream_unite(const StreamMerge *__restrict__ Mp) {
    const StreamMerge &M = *Mp;
    if (M.ctr->status & RUN_BAD) return;
    const long long P = M.ctr->punctures;
    const long long n_base = M.S->n;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < P; i += (long long)gridDim.x * NT) {
        const long long gi = n_base + i;
        // the run's component: its root is the slot of the run label
        const long long r = bsearch_ll(M.face, P, M.label[i]);
        if (r < 0) { atomicOr(&M.S->status, ST_PAIRING); continue; }
        if (r != i) uf_unite(M.gparent, (int)gi, (int)(n_base + r), &M.S->status);
        if (M.link_prev[i] >= 0) uf_unite(M.gparent, (int)gi, M.link_prev[i], &M.S->status);
    }
}

__global__ void __launch_bounds__(NT) k_stream_minima(const StreamMerge *__restrict__ Mp) {
    const StreamMerge &M = *Mp;
    if (M.ctr->status & RUN_BAD) return;
    const long long P = M.ctr->punctures;
    const long long n_base = M.S->n;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < P; i += (long long)gridDim.x * NT) {
        const long long gi = n_base + i;
        const int root = uf_find(M.gparent, (int)gi, &M.S->status);
        if (M.link_prev[i] >= 0) atomicMin(&M.gmin[root], M.gmin[M.old_root[i]]);
        else atomicMin(&M.gmin[root], M.gfid[gi]);
    }
}

// Ordered compaction of the delta (non-shadow) records with their
// provisional labels, and of the last-slice ordinal faces, in three passes
// over blocks of DELTA_BLOCK punctures: per-block counts, a scan of the block
// counts, per-block writes.  Then the report to the host and the advance of
// the stream's scalars.
__device__ __forceinline__ void delta_flags(const StreamMerge &M, long long k, long long n_base, long long i,
                                            long long P, int &keep, int &last) {
    keep = 0;
    last = 0;
    if (i < P) {
        keep = M.gshadow[n_base + i] ? 0 : 1;
        last = k == 0 ? 1 : (M.face[i] / M.T >= M.slice_verts ? 1 : 0);
    }
}

__global__ void __launch_bounds__(NT) k_delta_count(const StreamMerge *__restrict__ Mp) {
    const StreamMerge &M = *Mp;
    __shared__ long long red[NT / 32 + 1];
    if (M.ctr->status & RUN_BAD) return;
    const long long P = M.ctr->punctures;
    const long long k = M.S->k, n_base = M.S->n;
    const long long nb = (P + DELTA_BLOCK - 1) / DELTA_BLOCK;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        long long ck = 0, cl = 0;
        for (int o = threadIdx.x; o < DELTA_BLOCK; o += NT) {
            int keep, last;
            delta_flags(M, k, n_base, b * DELTA_BLOCK + o, P, keep, last);
            ck += keep;
            cl += last;
        }
        long long tk, tl;
        block_excl_scan<long long>(ck, red, tk);
        block_excl_scan<long long>(cl, red, tl);
        if (threadIdx.x == 0) {
            M.blk[b] = tk;
            M.blk[nb + b] = tl;
        }
    }
}

__global__ void __launch_bounds__(NT) k_delta_scan(const StreamMerge *__restrict__ Mp) {
    const StreamMerge &M = *Mp;
    __shared__ long long red[NT / 32 + 1];
    if (M.ctr->status & RUN_BAD) return;
    const long long P = M.ctr->punctures;
    const long long nb = (P + DELTA_BLOCK - 1) / DELTA_BLOCK;
    long long run_k = 0, run_l = 0;
    for (long long b0 = 0; b0 < nb; b0 += NT) {
        const long long b = b0 + threadIdx.x;
        const long long ck = b < nb ? M.blk[b] : 0, cl = b < nb ? M.blk[nb + b] : 0;
        long long tk, tl;
        const long long ek = block_excl_scan<long long>(ck, red, tk);
        const long long el = block_excl_scan<long long>(cl, red, tl);
        if (b < nb) {
            M.blk[2 * nb + b] = run_k + ek;
            M.blk[3 * nb + b] = run_l + el;
        }
        run_k += tk;
        run_l += tl;
    }
}

__global__ void __launch_bounds__(NT) k_delta_write(const StreamMerge *__restrict__ Mp) {
    const StreamMerge &M = *Mp;
    __shared__ long long red[NT / 32 + 1];
    if (M.ctr->status & RUN_BAD) return;
    const long long P = M.ctr->punctures;
    const long long k = M.S->k, n_base = M.S->n;
    const int cp = (int)(k & 1);
    const long long nb = (P + DELTA_BLOCK - 1) / DELTA_BLOCK;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        long long run_d = M.blk[2 * nb + b], run_o = M.blk[3 * nb + b];
        for (int o0 = 0; o0 < DELTA_BLOCK; o0 += NT) {
            const long long i = b * DELTA_BLOCK + o0 + threadIdx.x;
            int keep, last;
            delta_flags(M, k, n_base, i, P, keep, last);
            long long td, to;
            const long long pd = run_d + block_excl_scan<long long>(keep, red, td);
            const long long po = run_o + block_excl_scan<long long>(last, red, to);
            if (keep) {
                const long long gi = n_base + i;
                ftk_cp r = M.grec[gi];
                r.label = M.gmin[uf_find(M.gparent, (int)gi, &M.S->status)];
                M.delta[pd] = r;
            }
            if (last) {
                M.ord_fid[cp][po] = M.gfid[n_base + i];
                M.ord_gi[cp][po] = (int)(n_base + i);
            }
            run_d += td;
            run_o += to;
        }
    }
}

// after a merged push: the run's incremental detect state becomes the input
// of the next push (a run that was not merged keeps the old state)
__global__ void __launch_bounds__(NT) k_state_commit(const StreamMerge *__restrict__ Mp) {
    const StreamMerge &M = *Mp;
    if (M.ctr->status & RUN_BAD) return;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < M.st_words; i += (long long)gridDim.x * NT)
        M.st_in[i] = M.st_out[i];
}

// one thread: the report to the host and the advance of the scalars (after
// every kernel of the push has read them)
__global__ void k_stream_advance(const StreamMerge *__restrict__ Mp) {
    const StreamMerge &M = *Mp;
    const unsigned run_status = M.ctr->status;
    const long long P = M.ctr->punctures;
    M.view->run_status = run_status;
    M.view->punctures = P;
    if (run_status & RUN_BAD) {
        M.view->status = 0;
        M.view->delta = 0;
        __threadfence_system();
        return;
    }
    const long long k = M.S->k;
    const long long nb = (P + DELTA_BLOCK - 1) / DELTA_BLOCK;
    const long long nd = nb ? M.blk[2 * nb + nb - 1] + M.blk[nb - 1] : 0;
    const long long no = nb ? M.blk[3 * nb + nb - 1] + M.blk[nb + nb - 1] : 0;
    M.view->status = M.S->status;
    M.view->delta = nd;
    M.S->n_ord[k & 1] = no;
    M.S->n += P;
    M.S->k = k + 1;
    M.S->status = 0;
    __threadfence_system();
}

__global__ void __launch_bounds__(NT) k_stream_copy(const StreamSrc *src, float *dst, long long n) {
    const float *p = src->ptr;
    const long long stride = (long long)gridDim.x * NT;
    // the vector path only when both ends are 16-byte aligned (the second
    // slice of a two-slice buffer is not, unless the slice size is a
    // multiple of 4 floats)
    if (((((uintptr_t)p) | ((uintptr_t)dst)) & 15u) == 0) {
        const long long n4 = n >> 2;
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n4; i += stride) d4[i] = p4[i];
        for (long long i = (n4 << 2) + blockIdx.x * (long long)NT + threadIdx.x; i < n; i += stride) dst[i] = p[i];
    } else {
        for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += stride) dst[i] = p[i];
    }
}

// rows of nx floats -> rows of pitch floats, the padding repeating column
// nx-1; one element per thread and step (coalesced, no dependent chain)
__device__ __forceinline__ void pad_rows(const float *__restrict__ src, float *__restrict__ dst, int nx, int pitch,
                                         long long rows) {
    const long long n = rows * pitch;
    const long long stride = (long long)gridDim.x * NT;
#pragma unroll 4
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += stride) {
        const long long r = i / pitch;
        const int x = (int)(i - r * pitch);
        dst[i] = __ldg(src + r * nx + (x < nx ? x : nx - 1));
    }
}

__global__ void __launch_bounds__(NT) k_pad_rows(const float *src, float *dst, int nx, int pitch, long long rows) {
    pad_rows(src, dst, nx, pitch, rows);
}

__global__ void __launch_bounds__(NT) k_stream_copy_pad(const StreamSrc *src, float *dst, int nx, int pitch,
                                                        long long rows) {
    pad_rows(src->ptr, dst, nx, pitch, rows);
}

__global__ void __launch_bounds__(NT) k_fill_pad(float *dst, int nx, int pitch, long long rows) {
    const int w = pitch - nx;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < rows * w; i += (long long)gridDim.x * NT) {
        const long long r = i / w;
        float *row = dst + r * pitch;
        row[nx + (int)(i - r * w)] = row[nx - 1];
    }
}

__global__ void __launch_bounds__(NT) k_stream_final(long long n, const int *gshadow, int *gparent, const long long *gmin,
                                                     const ftk_cp *grec, ftk_cp *out, long long *count,
                                                     unsigned *status) {
    __shared__ long long red[NT / 32 + 1];
    long long run = 0;
    for (long long b0 = 0; b0 < n; b0 += NT) {
        const long long i = b0 + threadIdx.x;
        const int keep = i < n && !gshadow[i];
        long long t;
        const long long p = run + block_excl_scan<long long>(keep, red, t);
        if (keep) {
            ftk_cp r = grec[i];
            r.label = gmin[uf_find(gparent, (int)i, status)];
            out[p] = r;
        }
        run += t;
    }
    if (threadIdx.x == 0) *count = run;
}

cudaError_t launch_stream_merge(const StreamMerge *dM, const StreamMerge &M, long long cap, cudaStream_t s) {
    // grid-stride kernels over at most cap punctures (the run's capacity)
    const int sg = sparse_grid();
    const int g = (int)std::max<long long>(1, std::min<long long>(sg, (cap + NT - 1) / NT));
    k_stream_place<<<g, NT, 0, s>>>(dM);
    k_stream_unite<<<g, NT, 0, s>>>(dM);
    k_stream_minima<<<g, NT, 0, s>>>(dM);
    k_delta_count<<<g, NT, 0, s>>>(dM);
    k_delta_scan<<<1, NT, 0, s>>>(dM);
    k_delta_write<<<g, NT, 0, s>>>(dM);
    k_stream_advance<<<1, 1, 0, s>>>(dM);
    if (M.st_words > 0) k_state_commit<<<sg, NT, 0, s>>>(dM);
    return cudaGetLastError();
}

cudaError_t launch_stream_copy(const StreamSrc *src, float *dst, int nx, int pitch, long long rows, cudaStream_t s) {
    const int sg = sparse_grid();
    if (pitch == nx) {
        const long long n = (long long)nx * rows;
        const long long want = (n / 4 + NT - 1) / NT;
        k_stream_copy<<<(int)(want < sg ? (want > 0 ? want : 1) : sg), NT, 0, s>>>(src, dst, n);
    } else {
        const long long want = ((long long)pitch * rows + NT - 1) / NT;
        k_stream_copy_pad<<<(int)(want < 4LL * sg ? (want > 0 ? want : 1) : 4LL * sg), NT, 0, s>>>(src, dst, nx,
                                                                                                  pitch, rows);
    }
    return cudaGetLastError();
}

cudaError_t launch_pad_rows(const float *src, float *dst, int nx, int pitch, long long rows, cudaStream_t s) {
    const long long want = ((long long)pitch * rows + NT - 1) / NT;
    const long long cap = 4LL * sparse_grid();
    k_pad_rows<<<(int)(want < cap ? (want > 0 ? want : 1) : cap), NT, 0, s>>>(src, dst, nx, pitch, rows);
    return cudaGetLastError();
}

cudaError_t launch_fill_pad(float *dst, int nx, int pitch, long long rows, cudaStream_t s) {
    if (pitch > nx) k_fill_pad<<<sparse_grid(), NT, 0, s>>>(dst, nx, pitch, rows);
    return cudaGetLastError();
}

cudaError_t launch_stream_final(long long n, const int *gshadow, int *gparent, const long long *gmin,
                                const ftk_cp *grec, ftk_cp *out, long long *count, unsigned *status,
                                cudaStream_t s) {
    k_stream_final<<<1, NT, 0, s>>>(n, gshadow, gparent, gmin, grec, out, count, status);
    return cudaGetLastError();
}

thread_local const char *g_launch_stage = "";
const char *last_launch_stage() { return g_launch_stage; }

template <int N>
static cudaError_t launch_all(int variant, const Field &F, const Blocking &B, const Workspace &W, cudaStream_t s,
                              cudaEvent_t *ev) {
    const int sg = sparse_grid();
    // grid of a grid-stride kernel: at most `limit` blocks, and no more than
    // its work bound (the capacity of the list it walks) needs -- small
    // fields (batches, streamed slabs) launch few blocks
    auto gsize = [](int limit, long long items, int per_block) -> unsigned {
        const long long need = (items + per_block - 1) / per_block;
        return (unsigned)std::max<long long>(1, std::min<long long>(limit, need));
    };
    if (ev) cudaEventRecord(ev[0], s);
    // kernel attributes are set outside stream capture (a first, uncaptured
    // launch of the same shape always precedes a captured one)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (N == 3 && variant != VAR_TILE) {
        const cudaError_t e = launch_detect3(variant, F, B, W, s, capturing);
        if (e != cudaSuccess) return e;
    } else if (N == 2 && variant != VAR_TILE) {
        const cudaError_t e = launch_detect2(variant, F, B, W, s, capturing);
        if (e != cudaSuccess) return e;
    } else {
        const size_t smem = detect_smem_bytes(N, F, B);
        const cudaError_t e = raise_smem_cap((const void *)k_detect<N>, smem, capturing);
        if (e != cudaSuccess) return e;
        const long long units = (long long)B.ntc * B.nyb * B.nzb * (B.nxb > 1 ? B.nxb : 1);
        k_detect<N><<<(unsigned)units, NT, smem, s>>>(F, B, W);
    }
    if (ev) cudaEventRecord(ev[1], s);
    const bool stream = variant != VAR_TILE;
    if (stream) {
        if constexpr (N == 2)
            k_survive_eval_thread<N><<<gsize(resident_grid<k_survive_eval_thread<N>>(), W.scap, NT), NT, 0, s>>>(F, W);
        else k_survive_eval3<<<gsize(sg * 2, W.scap, NT / 16), NT, 0, s>>>(F, W);
        k_survive_scan<<<gsize(sg, W.scap, LB_TILE), NT, 0, s>>>(W);
    }
    {
        cudaError_t e2 = cudaGetLastError();
        if (e2 != cudaSuccess) { g_launch_stage = "detect/survive"; return e2; }
    }
    if (stream) k_seg_scan<<<(unsigned)std::min<long long>(sg, (W.nseg + SEG_TILE - 1) / SEG_TILE), NT, 0, s>>>(W);
    else k_scan<<<1, NT, 0, s>>>(W);
    if (ev) cudaEventRecord(ev[2], s);
    if (stream) {
        k_emit<N><<<gsize(resident_grid<k_emit<N>>(), W.scap, NT), NT, 0, s>>>(F, B, W);
        // few, long-running threads in 3D: small blocks spread them over every SM
        if constexpr (N == 3) {
            k_locate3<<<gsize(sg * 2, W.cap, NT / 4), NT, 0, s>>>(F, W);
            k_classify_exact<N><<<gsize(sg, W.cap, NT), NT, 0, s>>>(F, W);
        } else {
            k_locate<N><<<gsize(resident_grid<k_locate<N>>(), W.cap, NT), NT, 0, s>>>(F, W);
        }
    } else {
        k_finalize<N><<<sg, NT, 0, s>>>(F, B, W);
    }
    if (ev) cudaEventRecord(ev[3], s);
    if (stream) k_link_survivors<N><<<gsize(resident_grid<k_link_survivors<N>>(), W.scap * (N + 1), NT), NT, 0, s>>>(F, B, W);
    else k_link<N><<<sg, NT, 0, s>>>(F, B, W);
    if (ev) cudaEventRecord(ev[4], s);
    if (W.uf_limit < UF_LIMIT)
        k_label<N, true><<<gsize(resident_grid<k_label<N, true>>(), W.cap, NT), NT, 0, s>>>(F, W, stream ? 1 : 0);
    else
        k_label<N, false><<<gsize(resident_grid<k_label<N, false>>(), W.cap, NT), NT, 0, s>>>(F, W, stream ? 1 : 0);
    if (ev) cudaEventRecord(ev[5], s);
    cudaError_t e3 = cudaGetLastError();
    if (e3 != cudaSuccess) g_launch_stage = "scan..label";
    return e3;
}

cudaError_t launch_pipeline(int ndim, int variant, const Field &F, const Blocking &B, const Workspace &W,
                            cudaStream_t s, cudaEvent_t *ev) {
    g_launch_stage = "memset";
    cudaError_t e = cudaMemsetAsync(W.ctr, 0, sizeof(RunCounters), s);
    if (e != cudaSuccess) return e;
    g_launch_stage = "launch";
    Workspace Wl = W;
    Wl.uf_limit = uf_limit();
    return ndim == 2 ? launch_all<2>(variant, F, B, Wl, s, ev) : launch_all<3>(variant, F, B, Wl, s, ev);
}

}  // namespace ftk

// ----------------------------------------------------------------------------
// Trajectories as ordered polylines, and their slices at a time t (paper
// Sec. 4.1: a trajectory is a PL curve through spacetime that can be sliced
// at t = t0; Sec. 3.2).  Two punctured sides of one cell are consecutive
// points of a trajectory: inside the cell the interpolated field is linear,
// so its zero set is the segment between them.  Every face lies in at most
// two cells, so each puncture has at most two neighbours and a trajectory is
// a path or a closed loop.
// ----------------------------------------------------------------------------
namespace ftk {

// start of a trajectory without ends (a loop): the bytes 0x7f of a memset,
// above every puncture index
constexpr int TRAJ_NO_END = 0x7f7f7f7f;

// index of face id key in the sorted puncture array, or -1
__device__ __forceinline__ long long find_face(const long long *face, long long P, long long key) {
    long long lo = 0, hi = P;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (face[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < P && face[lo] == key) ? lo : -1;
}

// per puncture i: the punctured partner in each cell containing it (the
// cell's other punctured side), nbr[2i] <= nbr[2i+1], -1 for none
template <int N>
__global__ void __launch_bounds__(NT) k_traj_edges(Field F, Workspace W, int *nbr) {
    constexpr int D = N + 1;
    constexpr int FULL = (1 << D) - 1;
    const long long P = W.ctr->punctures;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < P; i += (long long)gridDim.x * NT) {
        const long long fid = W.face[i];
        int tt;
        const Pt base = decode_face<N>(F, fid, tt);
        int m[N];
        for (int k = 0; k < N; ++k) m[k] = mesh<N>().face[tt][k];
        Pt cb[2];
        int cm[2][D];
        int ncell = 0;
        if (m[N - 1] == FULL) {
            int prev = 0;
            for (int j = 0; j < N; ++j) {
                const int step = m[j] ^ prev;
                if (__popc(step) == 2) {
                    for (int a = 0; a < D; ++a) {
                        if (!((step >> a) & 1)) continue;
                        for (int q = 0; q < j; ++q) cm[ncell][q] = m[q];
                        cm[ncell][j] = prev | (1 << a);
                        for (int q = j; q < N; ++q) cm[ncell][q + 1] = m[q];
                        cb[ncell] = base;
                        ++ncell;
                    }
                    break;
                }
                prev = m[j];
            }
        } else {
            const int a = __ffs(FULL ^ m[N - 1]) - 1;
            const int ca = a == N ? 3 : a;
            const int ext = a == N ? F.nt : (a == 0 ? F.nx : a == 1 ? F.ny : F.nz);
            if (base.c[ca] >= 1) {
                cb[ncell] = base;
                cb[ncell].c[ca] -= 1;
                cm[ncell][0] = 1 << a;
                for (int q = 0; q < N; ++q) cm[ncell][q + 1] = m[q] | (1 << a);
                ++ncell;
            }
            if (base.c[ca] + 1 < ext) {
                cb[ncell] = base;
                for (int q = 0; q < N; ++q) cm[ncell][q] = m[q];
                cm[ncell][N] = FULL;
                ++ncell;
            }
        }
        int out[2] = {-1, -1};
        for (int c = 0; c < ncell; ++c) {
            for (int k = 0; k <= D; ++k) {
                Pt sb = cb[c];
                int sm[N];
                if (k == 0) {
                    sb = add_mask<N>(cb[c], cm[c][0]);
                    for (int q = 0; q < N; ++q) sm[q] = cm[c][q + 1] ^ cm[c][0];
                } else if (k == D) {
                    for (int q = 0; q < N; ++q) sm[q] = cm[c][q];
                } else {
                    int w = 0;
                    for (int q = 0; q < D; ++q)
                        if (q != k - 1) sm[w++] = cm[c][q];
                }
                const long long sid = face_id_of<N>(F, sb, sm);
                if (sid == fid) continue;
                const long long j = find_face(W.face, P, sid);
                if (j >= 0) out[c] = (int)j;
            }
        }
        if (out[0] > out[1]) { const int t = out[0]; out[0] = out[1]; out[1] = t; }
        nbr[2 * i] = out[0];
        nbr[2 * i + 1] = out[1];
    }
}

// per puncture: the index of its trajectory's root (the face with the
// smallest id, its label), the trajectory's size, and its smallest end
// (a puncture with fewer than two neighbours; TRAJ_NO_END for a loop)
__global__ void __launch_bounds__(NT) k_traj_roots(Workspace W, const int *nbr, int *root, int *size, int *start) {
    const long long P = W.ctr->punctures;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < P; i += (long long)gridDim.x * NT) {
        const long long r = find_face(W.face, P, W.label[i]);
        root[i] = (int)r;
        if (r < 0) {
            atomicOr(&W.ctr->status, ST_PAIRING);
            continue;
        }
        atomicAdd(&size[r], 1);
        if (nbr[2 * i] < 0) atomicMin(&start[r], (int)i);
    }
}

// Exclusive scan of v[0..n) into out[0..n], out[n] = total, in three
// passes over SCAN_BLOCKS chunks: block sums, one block scanning the sums
// (sums[nb] = total), and each block rescanning its chunk from its sum.
constexpr int SCAN_BLOCKS = 1024;
__global__ void __launch_bounds__(NT) k_scan_sums(const int *v, long long n, long long per, long long *sums) {
    __shared__ long long red[NT / 32 + 1];
    const long long a = blockIdx.x * per, b = min(n, a + per);
    long long loc = 0;
    for (long long i = a + threadIdx.x; i < b; i += NT) loc += v[i];
    long long tot;
    block_excl_scan<long long>(loc, red, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}
__global__ void __launch_bounds__(NT) k_scan_top(long long *sums, int nb) {
    __shared__ long long red[NT / 32 + 1];
    constexpr int PER = SCAN_BLOCKS / NT;
    long long loc[PER], s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = threadIdx.x * PER + k;
        loc[k] = i < nb ? sums[i] : 0;
        s += loc[k];
    }
    long long tot;
    long long ex = block_excl_scan<long long>(s, red, tot);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = threadIdx.x * PER + k;
        if (i < nb) sums[i] = ex;
        ex += loc[k];
    }
    if (threadIdx.x == 0) sums[nb] = tot;
}
__global__ void __launch_bounds__(NT) k_scan_apply(const int *v, long long n, long long per, const long long *sums,
                                                    int nb, long long *out) {
    __shared__ long long red[NT / 32 + 1];
    const long long a = blockIdx.x * per, b = min(n, a + per);
    long long run = sums[blockIdx.x];
    for (long long i0 = a; i0 < b; i0 += NT) {
        const long long i = i0 + threadIdx.x;
        const long long x = i < b ? v[i] : 0;
        long long tot;
        const long long ex = block_excl_scan<long long>(x, red, tot);
        if (i < b) out[i] = run + ex;
        run += tot;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[nb];
}

// the three passes (sums: SCAN_BLOCKS + 1 scratch values)
static void scan_ints(const int *v, long long n, long long *out, long long *sums, cudaStream_t s) {
    const long long nb = std::max<long long>(1, std::min<long long>(SCAN_BLOCKS, (n + 2047) / 2048));
    const long long per = (n + nb - 1) / nb;
    k_scan_sums<<<(unsigned)nb, NT, 0, s>>>(v, n, per, sums);
    k_scan_top<<<1, NT, 0, s>>>(sums, (int)nb);
    k_scan_apply<<<(unsigned)nb, NT, 0, s>>>(v, n, per, sums, (int)nb, out);
}

// sizes of the trajectories at their roots (0 elsewhere), for the scan of
// the trajectories' offsets; ones at the roots for their numbering
__global__ void __launch_bounds__(NT) k_traj_root_sizes(Workspace W, const int *root, const int *size, int *rsize,
                                                         int *isroot, int *maxlen) {
    const long long P = W.ctr->punctures;
    int mx = 0;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < P; i += (long long)gridDim.x * NT) {
        const bool r = root[i] == (int)i;
        rsize[i] = r ? size[i] : 0;
        isroot[i] = r ? 1 : 0;
        mx = r && size[i] > mx ? size[i] : mx;
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(maxlen, mx);
}

// Ordering the points of every trajectory, all points at once (list
// ranking by pointer jumping).  A loop is first cut open between its root
// (smallest index) and the root's larger neighbour, so that every
// trajectory is a path that starts at its smaller end: the order a walk
// from that end would give (a loop: from the root towards its smaller
// neighbour).  A state (node, prev, dist, ended) per point and direction d
// (first step to partner d) covers 2^k steps after round k; joining it with
// the state of the node it reached, in the direction that does not step
// back, doubles that.  ceil(log2(longest trajectory)) rounds end every walk
// at an end of its path; the distance to the smaller end is the rank.

// partners with every loop cut open: the slot of a loop root that holds its
// larger neighbour, and that neighbour's slot holding the root, become -1
// (one slot each, also when two cells join the same two points)
__global__ void __launch_bounds__(NT) k_traj_cut(Workspace W, const int *nbr, const int *root, const int *start,
                                                  int *nb2) {
    const long long P = W.ctr->punctures;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < P; i += (long long)gridDim.x * NT) {
        const int a = nbr[2 * i], b = nbr[2 * i + 1];
        int o0 = a, o1 = b;
        if (root[i] == (int)i && start[i] == TRAJ_NO_END) {
            // i is a loop root: cut its larger neighbour (slot 1: sorted)
            o1 = -1;
        }
        // a neighbour j that is a loop root with i as its larger neighbour
        if (b >= 0 && o1 >= 0 && root[b] == b && start[b] == TRAJ_NO_END && nbr[2 * b + 1] == (int)i) o1 = -1;
        else if (a >= 0 && root[a] == a && start[a] == TRAJ_NO_END && nbr[2 * a + 1] == (int)i) o0 = -1;
        nb2[2 * i] = o0;
        nb2[2 * i + 1] = o1;
    }
}

__global__ void __launch_bounds__(NT) k_traj_rank_init(Workspace W, const int *nb2, int4 *S) {
    const long long P = W.ctr->punctures;
    for (long long q = blockIdx.x * (long long)NT + threadIdx.x; q < 2 * P; q += (long long)gridDim.x * NT) {
        const int i = (int)(q >> 1), j = nb2[q];
        S[q] = j >= 0 ? make_int4(j, i, 1, 0) : make_int4(i, -1, 0, 1);
    }
}

__global__ void __launch_bounds__(NT) k_traj_rank_step(Workspace W, const int *nb2, const int4 *Sin, int4 *Sout) {
    const long long P = W.ctr->punctures;
    for (long long q = blockIdx.x * (long long)NT + threadIdx.x; q < 2 * P; q += (long long)gridDim.x * NT) {
        const int4 s = Sin[q];
        if (s.w) {
            Sout[q] = s;
            continue;
        }
        const int y = s.x, py = s.y;
        const int dy = nb2[2 * y] == py ? 1 : 0;     // the direction at y that does not step back
        const int4 t = Sin[2 * (long long)y + dy];
        Sout[q] = make_int4(t.x, t.z == 0 ? py : t.y, s.z + t.z, t.w);
    }
}

// every point at its rank in its trajectory's range; the roots also write
// the trajectory's offset and loop flag
__global__ void __launch_bounds__(NT) k_traj_place(Workspace W, const int4 *S, const int *root, const int *size,
                                                    const int *start, const long long *off, const long long *tidx,
                                                    int *order, long long *toff, uint8_t *closed, int *tpt) {
    const long long P = W.ctr->punctures;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < P; i += (long long)gridDim.x * NT) {
        const int4 s0 = S[2 * i], s1 = S[2 * i + 1];
        const int r = root[i];
        if (r < 0 || !s0.w || !s1.w) {                 // a walk that did not end: not a path
            atomicOr(&W.ctr->status, ST_PAIRING);
            continue;
        }
        const int first = min(s0.x, s1.x);            // the path's smaller end
        const int rank = s0.x == first ? s0.z : s1.z;
        const long long t = tidx[r];
        if (rank >= size[r] || s0.z + s1.z + 1 != size[r]) {   // not one path through all its points
            atomicOr(&W.ctr->status, ST_PAIRING);
            continue;
        }
        order[off[r] + rank] = (int)i;
        tpt[off[r] + rank] = (int)t;
        if (r == (int)i) {
            toff[t] = off[r];
            closed[t] = start[r] == TRAJ_NO_END ? 1 : 0;
        }
    }
}

// the records in trajectory, then path order
__global__ void __launch_bounds__(NT) k_traj_gather(Workspace W, const int *order, ftk_cp *rec) {
    const long long P = W.ctr->punctures;
    for (long long k = blockIdx.x * (long long)NT + threadIdx.x; k < P; k += (long long)gridDim.x * NT)
        rec[k] = W.packed[order[k]];
}

// time (grid units) of a puncture record
__device__ __forceinline__ double rec_t(const ftk_cp &r) { return (double)r.base[3] + (double)r.off[3]; }
__device__ __forceinline__ double rec_c(const ftk_cp &r, int a) { return (double)r.base[a] + (double)r.off[a]; }

// a double as an unsigned key of the same order (sign bit set: every bit
// flipped; else the sign bit set)
__device__ __forceinline__ unsigned long long order_key(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : u | 0x8000000000000000ull;
}
__device__ __forceinline__ double key_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? k & 0x7fffffffffffffffull : ~k));
}

// extents preset: smallest key = the largest key, largest = the smallest
__global__ void __launch_bounds__(NT) k_traj_ext_init(unsigned long long *ext, long long ntraj) {
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < ntraj; t += (long long)gridDim.x * NT) {
        ext[2 * t] = ~0ull;
        ext[2 * t + 1] = 0ull;
    }
}

// per point: its trajectory's smallest and largest point time (keys, ext[2t]
// and ext[2t + 1], preset to the largest and smallest key)
__global__ void __launch_bounds__(NT) k_traj_extent(const ftk_cp *rec, const int *tpt, long long P,
                                                     unsigned long long *ext) {
    for (long long k = blockIdx.x * (long long)NT + threadIdx.x; k < P; k += (long long)gridDim.x * NT) {
        const unsigned long long key = order_key(rec_t(rec[k]));
        const long long t = tpt[k];
        atomicMin(&ext[2 * t], key);
        atomicMax(&ext[2 * t + 1], key);
    }
}

// Post-processing of the trajectories (paper Sec. 4.2, filtering and type
// smoothing).  Per trajectory: kept iff its time extent (largest minus
// smallest point time) is at least min_duration, it has at least min_points
// points and it is not a loop when loops are dropped.
__global__ void __launch_bounds__(NT) k_traj_keep(const unsigned long long *ext, const long long *toff,
                                                   const uint8_t *closed, long long ntraj, double min_duration,
                                                   long long min_points, int drop_loops, int *kept_size,
                                                   int *kept_one) {
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < ntraj; t += (long long)gridDim.x * NT) {
        const long long n = toff[t + 1] - toff[t];
        const double lo = key_value(ext[2 * t]), hi = key_value(ext[2 * t + 1]);
        const bool keep = n >= min_points && hi - lo >= min_duration && !(drop_loops && closed[t]);
        kept_size[t] = keep ? (int)n : 0;
        kept_one[t] = keep ? 1 : 0;
    }
}

// Copies the kept trajectories to their new offsets; with h > 0 a point's
// Morse index is replaced by the common index of the h points before and
// the h points after it along the path when those 2h points all agree and
// it differs (loops wrap around; on a path, points with fewer than h
// neighbours on a side keep theirs).  Every decision reads the original
// indices.
__global__ void __launch_bounds__(NT) k_traj_compact(const ftk_cp *rec, const long long *toff, const uint8_t *closed,
                                                      const int *tpt, long long P, int h, const long long *noff,
                                                      const long long *nidx, const int *kept_one, ftk_cp *out,
                                                      long long *out_off, uint8_t *out_closed) {
    for (long long pk = blockIdx.x * (long long)NT + threadIdx.x; pk < P; pk += (long long)gridDim.x * NT) {
        const int t = tpt[pk];
        if (!kept_one[t]) continue;
        const long long a0 = toff[t], n = toff[t + 1] - a0;
        const long long o = noff[t], j = pk - a0;
        if (j == 0) {
            out_off[nidx[t]] = o;
            out_closed[nidx[t]] = closed[t];
        }
        const bool loop = closed[t] != 0;
        {
            ftk_cp r = rec[a0 + j];
            if (h > 0 && (loop ? n > 2 * (long long)h : (j >= h && j + h < n))) {
                const long long jm = (j - 1 + n) % n;
                const int8_t ref = rec[a0 + jm].morse_index;
                bool same = true;
                for (int q = 1; q <= h && same; ++q) {
                    same &= rec[a0 + (j - q + n) % n].morse_index == ref;
                    same &= rec[a0 + (j + q) % n].morse_index == ref;
                }
                if (same && ref != r.morse_index) r.morse_index = ref;
            }
            out[o + j] = r;
        }
    }
}

// segments (consecutive points in path order, and the closing segment of a
// loop) that cross time t0: t_a <= t0 < t_b or t_b <= t0 < t_a, one thread
// per segment, named by its first point k in record order.  Pass 1 flags
// the crossing segments; pass 2 writes the crossing points at the flags'
// scan (so in trajectory, then path order), interpolated linearly in time
// along the segment.
__global__ void __launch_bounds__(NT) k_traj_slice(const ftk_cp *rec, const long long *toff, const uint8_t *closed,
                                                    const int *tpt, long long P, double t0, int *cnt,
                                                    const long long *soff, ftk_slice_point *pts) {
    for (long long k = blockIdx.x * (long long)NT + threadIdx.x; k < P; k += (long long)gridDim.x * NT) {
        const int t = tpt[k];
        const long long a0 = toff[t], n = toff[t + 1] - a0, j = k - a0;
        const long long nseg = closed[t] ? n : n - 1;
        bool hit = false;
        if (j < nseg) {
            const ftk_cp &A = rec[k];
            const ftk_cp &B = rec[j + 1 == n ? a0 : k + 1];
            const double ta = rec_t(A), tb = rec_t(B);
            hit = (ta <= t0 && t0 < tb) || (tb <= t0 && t0 < ta);
            if (hit && pts) {
                const double s = (t0 - ta) / (tb - ta);
                ftk_slice_point p;
                p.label = A.label;
                p.face_a = A.face_id < B.face_id ? A.face_id : B.face_id;
                p.face_b = A.face_id < B.face_id ? B.face_id : A.face_id;
                for (int a = 0; a < 3; ++a) p.pos[a] = rec_c(A, a) + s * (rec_c(B, a) - rec_c(A, a));
                pts[soff[k]] = p;
            }
        }
        if (!pts) cnt[k] = hit ? 1 : 0;
    }
}

}  // namespace ftk

namespace ftk {

cudaError_t launch_trajectories(int ndim, const Field &F, const Workspace &W, long long P, const TrajBuffers &T,
                                cudaStream_t s, long long *ntraj, int *maxlen) {
    const int grid = sparse_grid();
    cudaError_t e;
    if (ndim == 2) k_traj_edges<2><<<grid, NT, 0, s>>>(F, W, T.nbr);
    else k_traj_edges<3><<<grid, NT, 0, s>>>(F, W, T.nbr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(T.size, 0, sizeof(int) * P, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(T.start, 0x7f, sizeof(int) * P, s)) != cudaSuccess) return e;   // TRAJ_NO_END
    k_traj_roots<<<grid, NT, 0, s>>>(W, T.nbr, T.root, T.size, T.start);
    if ((e = cudaMemsetAsync(T.maxlen, 0, sizeof(int), s)) != cudaSuccess) return e;
    k_traj_root_sizes<<<grid, NT, 0, s>>>(W, T.root, T.size, T.rsize, T.isroot, T.maxlen);
    scan_ints(T.rsize, P, T.off, T.scan, s);
    scan_ints(T.isroot, P, T.tidx, T.scan, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(ntraj, T.tidx + P, sizeof(long long), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(maxlen, T.maxlen, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t launch_traj_walk(const Workspace &W, long long P, long long ntraj, long long maxlen, const TrajBuffers &T,
                             cudaStream_t s) {
    const int g = resident_grid<k_traj_rank_step>();
    k_traj_cut<<<g, NT, 0, s>>>(W, T.nbr, T.root, T.start, T.nb2);
    k_traj_rank_init<<<g, NT, 0, s>>>(W, T.nb2, T.rk[0]);
    int cur = 0;
    for (long long span = 1; span < maxlen; span *= 2) {
        k_traj_rank_step<<<g, NT, 0, s>>>(W, T.nb2, T.rk[cur], T.rk[cur ^ 1]);
        cur ^= 1;
    }
    k_traj_place<<<g, NT, 0, s>>>(W, T.rk[cur], T.root, T.size, T.start, T.off, T.tidx, T.order, T.toff, T.closed,
                                  T.tpt);
    k_traj_gather<<<resident_grid<k_traj_gather>(), NT, 0, s>>>(W, T.order, T.rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(T.toff + ntraj, T.off + P, sizeof(long long), cudaMemcpyDeviceToDevice, s);
}

cudaError_t launch_traj_slice(const TrajBuffers &T, long long P, double t0, int *cnt, long long *soff,
                              ftk_slice_point *pts, cudaStream_t s) {
    k_traj_slice<<<resident_grid<k_traj_slice>(), NT, 0, s>>>(T.rec, T.toff, T.closed, T.tpt, P, t0, cnt, soff, pts);
    if (!pts) scan_ints(cnt, P, soff, T.scan, s);
    return cudaGetLastError();
}

}  // namespace ftk

namespace ftk {

cudaError_t set_wait_limits(long long uf_steps, long long lookback_cycles) {
    const int u = uf_steps > 0 ? (int)std::min<long long>(uf_steps, UF_LIMIT) : UF_LIMIT;
    const long long c = lookback_cycles > 0 ? std::min<long long>(lookback_cycles, WAIT_CYCLES) : WAIT_CYCLES;
    g_host_uf_limit.store(u);
    return cudaMemcpyToSymbol(g_lookback_cycles, &c, sizeof(c));
}

int uf_limit() { return g_host_uf_limit.load(); }

}  // namespace ftk

namespace ftk {

cudaError_t launch_traj_filter(const TrajBuffers &T, long long P, long long ntraj, double min_duration,
                               long long min_points, int drop_loops, int h, unsigned long long *ext, int *kept_size,
                               int *kept_one, long long *noff, long long *nidx, cudaStream_t s) {
    k_traj_ext_init<<<sparse_grid(), NT, 0, s>>>(ext, ntraj);
    k_traj_extent<<<resident_grid<k_traj_extent>(), NT, 0, s>>>(T.rec, T.tpt, P, ext);
    k_traj_keep<<<sparse_grid(), NT, 0, s>>>(ext, T.toff, T.closed, ntraj, min_duration, min_points, drop_loops,
                                             kept_size, kept_one);
    scan_ints(kept_size, ntraj, noff, T.scan, s);
    scan_ints(kept_one, ntraj, nidx, T.scan, s);
    return cudaGetLastError();
}

cudaError_t launch_traj_compact(const TrajBuffers &T, long long P, int h, const long long *noff,
                                const long long *nidx, const int *kept_one, ftk_cp *out, long long *out_off,
                                uint8_t *out_closed, cudaStream_t s) {
    k_traj_compact<<<resident_grid<k_traj_compact>(), NT, 0, s>>>(T.rec, T.toff, T.closed, T.tpt, P, h, noff, nidx,
                                                                  kept_one, out, out_off, out_closed);
    return cudaGetLastError();
}

}  // namespace ftk
