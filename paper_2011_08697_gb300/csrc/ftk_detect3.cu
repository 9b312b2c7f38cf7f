// Streaming sign cull for 3D fields (3D + time, paper Sec. 3.3 mesh, Sec. 4.1
// predicate): the dense, HBM-bound pass of the 3D pipeline.
//
// A unit (one CTA) owns ry cube rows (y) x rz cube planes (z) x tc base
// slices (t) of cubes, i.e. spacetime cubes whose base vertex lies in that
// block.  Warp roles:
//  * producer (one lane): per slice, rz + 3 plane chunks -- rows
//    y0-1 .. y0+ry+1 of planes z0-1 .. z0+rz+1, clamped to the grid, one
//    contiguous bulk copy each -- into a ring of smem slots (full / empty
//    mbarriers);
//  * consumer warps (four; eight for rows of 513-1024 floats, one per
//    chunk): warp w owns 4 G rows (y) of one 128-column chunk (4 columns
//    per lane) and walks the planes of each slice in z.  Each plane
//    chunk is read from shared memory once, right after it lands: the warp
//    loads its 4 rows plus one halo row on each side, quantises them
//    (F = rint(f 2^S) in a magic-number encoding, exact for |F| <= 2^22;
//    wider values flag an exact re-run) into registers and releases the
//    slot.  Three planes stay in registers (z-1, z, z+1; their roles rotate
//    with the walk, so nothing is copied), which gives the central
//    differences in x (neighbour lanes), y (halo rows) and z, packed as 12
//    sign bits per lane (G_r < 0; zero counts as positive) and kept twice
//    (an AND half and an OR half).  The cube words of two consecutive G
//    planes are combined in registers over z, then over y (the group's first
//    row comes from the next warp through shared memory, one named barrier
//    per plane), over x (neighbour lane) and over t (the previous slice's
//    cube words stay in smem).  A cube survives iff every gradient
//    component has corners of both signs; that test is exact, because the
//    symbolic perturbation is infinitesimal and adds a positive term to a
//    zero component.  Survivors go to a double-buffered smem bitmap;
//  * compactor warp: per base slice, turns the bitmap into ordered lists of
//    surviving cubes, one per segment (t, z, y-block), in global memory.
// Grid edges: clamped rows, planes and columns turn every one-sided
// difference into a doubled central difference of the same sign; a cube
// whose upper corners leave the grid repeats its lower corners (the faces it
// owns then lie in the grid's boundary).  Every wait is bounded; a wait that
// runs out sets a shared abort flag, every warp drains and the run reports
// ST_TIMEOUT.
#include <cuda_runtime.h>

#include <climits>

#include "ftk_kernels.cuh"
#include "ftk_tma.cuh"

namespace ftk {

namespace {

constexpr int S3_RPW = 4;                 // G rows per consumer warp
constexpr int S3_NS = 6;                  // smem ring slots (plane chunks)
constexpr float S3_RANGE = 268435456.0f;  // 2^28
constexpr uint32_t ALL = 0xffffffffu;

__host__ __device__ inline int s3_round16(int v) { return (v + 15) & ~15; }
// 128-column chunks per row (a power of two, so that the warps split evenly)
__host__ __device__ inline int s3_chunks(int nx) { return nx <= 128 ? 1 : nx <= 256 ? 2 : nx <= 512 ? 4 : 8; }
// consumer warps: four, stacked in y over the chunks, or one per chunk for
// rows of eight chunks
__host__ __device__ constexpr int s3_nw_of(int xc) { return xc > 4 ? xc : 4; }
__host__ __device__ inline int s3_nw(int nx) { return s3_nw_of(s3_chunks(nx)); }
__host__ __device__ inline int s3_threads(int nx) { return (s3_nw(nx) + 2) * 32; }
// G rows per unit: the consumer warps of one chunk stacked in y (ry + 1)
__host__ __device__ inline int s3_grows(int nx) { return s3_nw(nx) / s3_chunks(nx) * S3_RPW; }

struct S3Layout {
    int slot_floats, ring, bars, abort, xy, xx, ts, bm, rw, cnt, total;
};
__host__ __device__ inline S3Layout s3_layout(int nx, int ry, int rz) {
    constexpr int ns = S3_NS;
    S3Layout L;
    const int xc = s3_chunks(nx);
    const int gr = s3_grows(nx);
    L.slot_floats = (ry + 3) * nx;                 // nx % 4 == 0: a multiple of 16 bytes
    L.ring = 0;
    L.bars = L.ring + ns * L.slot_floats * 4;
    L.abort = L.bars + (2 * ns + 4) * 8;
    L.xy = s3_round16(L.abort + 4);                // [2][warps][32] z-paired words of a warp's first G row
    L.xx = L.xy + 2 * s3_nw(nx) * 32 * 4;          // [2][gr][xc] y-paired words of a chunk's first column
    L.ts = s3_round16(L.xx + 2 * gr * xc * 4);     // [rz][ry][xc][32] cube words of the previous slice
    L.bm = L.ts + rz * ry * xc * 32 * 4;
    L.rw = (ry * nx + 31) / 32;                    // bitmap words per cube plane
    L.cnt = L.bm + 2 * rz * L.rw * 4;              // [2][rz] survivor counts per cube plane
    L.total = s3_round16(L.cnt + 2 * rz * 4);
    return L;
}

// AND in the low half, OR in the high half
__device__ __forceinline__ uint32_t cmb(uint32_t a, uint32_t b) {
    return ((a & b) & 0x0000FFFFu) | ((a | b) & 0xFFFF0000u);
}

// bounded wait that also gives up once another warp has aborted; warps off
// the critical path back off with a sleep between polls (sleep_ns > 0) so
// that they leave the issue slots to the consumers
__device__ __forceinline__ bool wait_ab(uint64_t *bar, uint32_t parity, volatile int *abort, unsigned sleep_ns = 0) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort = 1;
            return false;
        }
        if (sleep_ns) __nanosleep(sleep_ns);
    }
    return true;
}

// quantised sample: fast form = bits of v 2^S + 1.5 2^23 (the float is the
// integer rint(v 2^S) + 1.5 2^23 exactly when |v 2^S| <= 2^22); exact form =
// rint(v 2^S) as a two's complement integer
template <bool EXACT>
__device__ __forceinline__ uint32_t q3(float v, float scale, uint32_t &bad) {
    if (EXACT) {
        const float w = v * scale;
        const bool in = fabsf(w) <= S3_RANGE;
        bad |= in ? 0u : 1u;
        return (uint32_t)(in ? __float2int_rn(w) : 0);
    }
    return __float_as_uint(__fmaf_rn(v, scale, MAGIC_F));
}
// bit 31 = sign of the integer difference a - b (zero is positive)
template <bool EXACT>
__device__ __forceinline__ uint32_t qd(uint32_t a, uint32_t b) {
    if (EXACT) return a - b;
    return __float_as_uint(__uint_as_float(a) - __uint_as_float(b));
}

// one plane chunk of one consumer lane, quantised: rows gr0-1 .. gr0+4 of
// the warp (clamped), 4 columns each, and (several chunks per row) the
// column beyond the chunk's edge on the edge lanes
template <int XC>
struct PlaneRegs {
    uint32_t v[S3_RPW + 2][4];
    uint32_t h[XC > 1 ? S3_RPW + 2 : 1];
};

template <bool EXACT, int XC>
__global__ void __launch_bounds__((s3_nw_of(XC) + 2) * 32, XC > 4 ? 1 : 2)
    k_detect3_stream(Field F, Blocking B, Workspace W) {
    constexpr int S3_NW = s3_nw_of(XC);    // consumer warps
    extern __shared__ __align__(128) unsigned char smem[];
    // the sweep covers the padded row (pitch columns, the padding repeating
    // column nx-1); survivors are the grid's (columns < nxl)
    const int nx = F.pitch, nxl = F.nx, ny = F.ny, nz = F.nz, nt = F.nt;
    const int RY = B.ry, RZ = B.rz;
    constexpr int NS = S3_NS;
    constexpr int NG = S3_NW / XC;         // warps stacked in y per chunk
    const S3Layout L = s3_layout(nx, RY, RZ);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *ring = reinterpret_cast<float *>(smem + L.ring);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint64_t *empty = full + NS;
    uint64_t *done = empty + NS;     // [2] slab bits complete (consumer warps arrive)
    uint64_t *freed = done + 2;      // [2] bitmap compacted and cleared (compactor arrives)
    volatile int *abort = reinterpret_cast<volatile int *>(smem + L.abort);
    uint32_t *XY = reinterpret_cast<uint32_t *>(smem + L.xy);
    uint32_t *XX = reinterpret_cast<uint32_t *>(smem + L.xx);
    uint32_t *TS = reinterpret_cast<uint32_t *>(smem + L.ts);
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem + L.bm);
    int *scnt = reinterpret_cast<int *>(smem + L.cnt);    // survivors per (buffer, cube plane)
    unsigned *status = &W.ctr->status;

    const int yb = blockIdx.x % B.nyb;
    const int rest = blockIdx.x / B.nyb;
    const int zb = rest % B.nzb;
    const int tci = rest / B.nzb;
    const int y0 = yb * RY, z0 = zb * RZ, t0 = tci * B.tc;
    const int t_end = min(nt, t0 + B.tc);
    const int s_last = min(t_end, nt - 1);
    const int nsl = s_last - t0 + 1;      // slices streamed
    const int nslab = t_end - t0;         // base slices owned
    const int PL = RZ + 3;                // plane chunks per slice
    const int J = nsl * PL;
    const int ylo = max(y0 - 1, 0), yhi = min(y0 + RY + 1, ny - 1);
    const int ncy = min(RY, ny - y0);     // cube rows present
    const int ncz = min(RZ, nz - z0);     // cube planes present
    const int GR = NG * S3_RPW;           // G rows per unit (RY + 1)

    if (threadIdx.x == 0) {
        for (int k = 0; k < NS; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], S3_NW);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&done[b], S3_NW);
            mbar_init(&freed[b], 1);
        }
        *abort = 0;
        mbar_fence_init();
    }
    for (int i = threadIdx.x; i < 2 * RZ * L.rw; i += blockDim.x) bm[i] = 0u;
    for (int i = threadIdx.x; i < 2 * RZ; i += blockDim.x) scnt[i] = 0;
    __syncthreads();

    if (warp == S3_NW) {
        // ---------------- producer ----------------------------------------
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)((yhi - ylo + 1) * nx * 4);
            int issued = 0, slot = 0;
            uint32_t phase = 0;              // parity of the slot's next empty phase, flipped per lap
            bool stop = false;
            for (int sl = 0; sl < nsl && !stop; ++sl) {
                const int s = t0 + sl;
                for (int k = 0; k < PL; ++k) {
                    if (issued >= NS && !wait_ab(&empty[slot], phase ^ 1u, abort, 64)) {
                        stop = true;
                        break;
                    }
                    const int z = min(max(z0 - 1 + k, 0), nz - 1);
                    const float *src = F.f + (((long long)s * nz + z) * ny + ylo) * nx;
                    mbar_arrive_expect_tx(&full[slot], bytes);
                    tma_row(ring + (size_t)slot * L.slot_floats, src, bytes, &full[slot]);
                    ++issued;
                    if (++slot == NS) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (issued < J) {
                atomicOr(status, ST_TIMEOUT);
                *abort = 1;
                // never leave a copy in flight into a CTA that is exiting
                for (int j = max(0, issued - NS); j < issued; ++j) mbar_wait(&full[j % NS], (j / NS) & 1);
            }
        }
        return;
    }
    if (warp == S3_NW + 1) {
        // ---------------- compactor ---------------------------------------
        for (int q = 0; q < nslab; ++q) {
            const int b = q & 1;
            if (!__all_sync(ALL, wait_ab(&done[b], (q >> 1) & 1, abort, 256))) {
                if (lane == 0) atomicOr(status, ST_TIMEOUT);
                return;
            }
            const int t = t0 + q;
            const float inv_nx = 1.0f / (float)nx;
            for (int ci = 0; ci < ncz; ++ci) {
                const int z = z0 + ci;
                const int total = scnt[b * RZ + ci];
                const long long seg = ((long long)t * nz + z) * B.nyb + yb;
                long long base = 0;
                if (lane == 0) {
                    base = total ? (long long)atomicAdd(&W.ctr->survivors, (unsigned long long)total) : 0;
                    W.seg_scnt[seg] = total;
                    W.seg_sstage[seg] = base;
                    if (base + total > W.scap) atomicOr(status, ST_SOVERFLOW);
                }
                if (total == 0) continue;   // warp-uniform; the words are all zero already
                base = __shfl_sync(ALL, base, 0);
                compact_bits<2>(bm + (b * RZ + ci) * L.rw, L.rw, nx, nxl, inv_nx, ((long long)t * nz + z) * ny + y0,
                                base, W.surv, W.scap);
            }
            __syncwarp();
            if (lane < RZ) scnt[b * RZ + lane] = 0;
            __syncwarp();
            if (lane == 0) mbar_arrive(&freed[b]);
        }
        return;
    }

    // ---------------- consumers ---------------------------------------------
    const int c = warp % XC;               // this warp's 128-column chunk
    const int grp = warp / XC;             // its place in the chunk's stack of warps
    const int gr0 = grp * S3_RPW;          // first G row (unit-relative)
    const int xb = c * 128 + lane * 4;     // first column of this lane
    const bool act = xb < nx;
    const int xa = act ? xb : 0;           // a safe address for idle lanes
    const bool xlast = act && xb + 4 >= nx;
    // the lane's columns inside the grid (the rest is padding)
    const uint32_t gmask = act ? (1u << max(0, min(4, nxl - xb))) - 1u : 0u;
    // halo sample of the edge lanes of a chunk: lane 0 the column left of the
    // chunk (itself at x = 0), lane 31 the column right of it (unused at the
    // grid's edge)
    const int hoff = !act ? 0 : lane == 0 ? (xa == 0 ? 0 : -1) : (lane == 31 && !xlast ? 4 : 0);
    // smem offsets (floats, within a plane chunk) of the warp's rows
    // gr0-1 .. gr0+4, clamped to the grid
    int ro[S3_RPW + 2];
#pragma unroll
    for (int i = 0; i < S3_RPW + 2; ++i) ro[i] = (min(max(y0 + gr0 - 1 + i, 0), ny - 1) - ylo) * nx + xa;
    // cube row gr0 + r steps to G row gr0 + r + 1 inside the grid; at the top
    // edge the cube repeats its own row
    uint32_t ystep = 0;
#pragma unroll
    for (int r = 0; r < S3_RPW; ++r) ystep |= (y0 + gr0 + r + 1 <= ny - 1 ? 1u : 0u) << r;
    const float scale = F.scale;
    uint32_t bad = 0, qa_and = 0xffffffffu, qa_or = 0u;
    bool ok = true;
    int xs = 0;                            // cube stages so far (parity of the exchange buffers)

    // plane chunk j into registers: wait for it, load and quantise the
    // warp's rows, release the slot
    auto load = [&](PlaneRegs<XC> &P, int j) {
        if (ok && !wait_ab(&full[j % NS], (j / NS) & 1, abort)) ok = false;
        ok = __all_sync(ALL, ok);
        if (ok) {
            const float *pc = ring + (size_t)(j % NS) * L.slot_floats;
#pragma unroll
            for (int i = 0; i < S3_RPW + 2; ++i) {
                const float4 v = *reinterpret_cast<const float4 *>(pc + ro[i]);
                P.v[i][0] = q3<EXACT>(v.x, scale, bad);
                P.v[i][1] = q3<EXACT>(v.y, scale, bad);
                P.v[i][2] = q3<EXACT>(v.z, scale, bad);
                P.v[i][3] = q3<EXACT>(v.w, scale, bad);
                if (XC > 1) P.h[i] = q3<EXACT>(pc[ro[i] + hoff], scale, bad);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[j % NS]);
    };

    // G sign words (12 bits: G_x, G_y, G_z of the lane's 4 columns, low to
    // high, in both halves) of the warp's 4 rows of plane Y, with the planes
    // below (M) and above (P) in z
    auto gwords = [&](const PlaneRegs<XC> &M, const PlaneRegs<XC> &Y, const PlaneRegs<XC> &P, uint32_t *w) {
#pragma unroll
        for (int r = 0; r < S3_RPW; ++r) {
            const uint32_t *o = Y.v[r + 1];
            const uint32_t up = __shfl_up_sync(ALL, o[3], 1);
            const uint32_t dn = __shfl_down_sync(ALL, o[0], 1);
            uint32_t lq, rq;
            if (XC > 1) {
                lq = lane == 0 ? Y.h[r + 1] : up;
                rq = xlast ? o[3] : lane == 31 ? Y.h[r + 1] : dn;
            } else {
                lq = lane == 0 ? o[0] : up;
                rq = xlast ? o[3] : dn;
            }
            if (!EXACT) {
                qa_and &= o[0] & o[1];
                qa_and &= o[2] & o[3];
                qa_or |= o[0] | o[1];
                qa_or |= o[2] | o[3];
            }
            // three independent 4-bit chains (short dependency chains), then
            // one combine: G_x in bits 0-3, G_y in 4-7, G_z in 8-11
            uint32_t gz = 0, gy = 0, gx = 0;
#pragma unroll
            for (int i = 3; i >= 0; --i) gz = __funnelshift_l(qd<EXACT>(P.v[r + 1][i], M.v[r + 1][i]), gz, 1);
#pragma unroll
            for (int i = 3; i >= 0; --i) gy = __funnelshift_l(qd<EXACT>(Y.v[r + 2][i], Y.v[r][i]), gy, 1);
            gx = __funnelshift_l(qd<EXACT>(rq, o[2]), gx, 1);
            gx = __funnelshift_l(qd<EXACT>(o[3], o[1]), gx, 1);
            gx = __funnelshift_l(qd<EXACT>(o[2], o[0]), gx, 1);
            gx = __funnelshift_l(qd<EXACT>(o[1], lq), gx, 1);
            const uint32_t g = gx | (gy << 4) | (gz << 8);
            w[r] = g | (g << 16);
        }
    };

    uint32_t prev[S3_RPW], cur[S3_RPW];

    // cube plane ci between G planes ci and ci + 1 (words prev, cur): combine
    // over z, y, x and t, emit survivors of base slice t0 + sl - 1
    auto cubes = [&](int ci, int sl, uint32_t *bq, int q) {
        const int par = xs & 1;
        ++xs;
        const bool zstep = z0 + ci + 1 <= nz - 1;   // else the cube repeats plane ci
        uint32_t zw[S3_RPW];
#pragma unroll
        for (int r = 0; r < S3_RPW; ++r) zw[r] = zstep ? cmb(prev[r], cur[r]) : prev[r];
        XY[(par * S3_NW + warp) * 32 + lane] = zw[0];
        named_sync(1, S3_NW * 32);
        const uint32_t below = grp + 1 < NG ? XY[(par * S3_NW + warp + XC) * 32 + lane] : 0u;
        uint32_t yw[S3_RPW];
#pragma unroll
        for (int r = 0; r < S3_RPW; ++r) {
            const uint32_t nxt = r + 1 < S3_RPW ? zw[r + 1] : below;
            yw[r] = (ystep >> r) & 1u ? cmb(zw[r], nxt) : zw[r];
        }
        if (XC > 1) {
            if (lane == 0)
#pragma unroll
                for (int r = 0; r < S3_RPW; ++r) XX[(par * GR + gr0 + r) * XC + c] = yw[r];
            named_sync(1, S3_NW * 32);
        }
        int nsv = 0;
#pragma unroll
        for (int r = 0; r < S3_RPW; ++r) {
            const int cr = gr0 + r;
            if (cr >= ncy) break;              // warp-uniform
            const uint32_t u = yw[r];
            // the cube's x+1 corners: the next lane's first column
            uint32_t nxt = __shfl_down_sync(ALL, u, 1);
            if (XC > 1 && lane == 31 && c + 1 < XC) nxt = XX[(par * GR + cr) * XC + c + 1];
            uint32_t nb = ((u >> 1) & 0x07770777u) | ((nxt & 0x01110111u) << 3);
            if (xlast) nb = (nb & ~0x08880888u) | (u & 0x08880888u);   // column nx-1
            const uint32_t Pw = cmb(u, nb);
            uint32_t *ts = TS + ((ci * RY + cr) * XC + c) * 32 + lane;
            if (sl >= 1) {
                const uint32_t c4 = cmb(Pw, *ts);
                const uint32_t mixed = (c4 >> 16) & ~c4 & 0xFFFu;
                const uint32_t sv = mixed & (mixed >> 4) & (mixed >> 8) & gmask;
                if (sv) {
                    const int idx = cr * nx + xb;
                    atomicOr(&bq[ci * L.rw + (idx >> 5)], sv << (idx & 31));
                    nsv += __popc(sv);
                }
            }
            *ts = Pw;
        }
        if (sl >= 1) {
            nsv = __reduce_add_sync(ALL, nsv);
            if (lane == 0 && nsv) atomicAdd(&scnt[(q & 1) * RZ + ci], nsv);
        }
    };

    PlaneRegs<XC> A, Bp, C;
    for (int sl = 0; sl < nsl; ++sl) {
        const int q = sl - 1;              // slab completed by this slice
        const int jb = sl * PL;
        uint32_t *bq = bm + (q & 1) * RZ * L.rw;
        if (ok && q >= 2 && !wait_ab(&freed[q & 1], ((q >> 1) - 1) & 1, abort)) ok = false;
        ok = __all_sync(ALL, ok);
        load(A, jb);
        load(Bp, jb + 1);
        load(C, jb + 2);
        // G planes gi = 0 .. RZ; planes M, Y, P rotate through A, Bp, C
        auto step = [&](PlaneRegs<XC> &M, PlaneRegs<XC> &Y, PlaneRegs<XC> &P, int gi) {
            if (ok) gwords(M, Y, P, cur);
            if (gi >= 1 && gi - 1 < ncz) cubes(gi - 1, sl, bq, q);
#pragma unroll
            for (int r = 0; r < S3_RPW; ++r) prev[r] = cur[r];
            if (gi + 3 < PL) load(M, jb + gi + 3);
        };
        for (int gi = 0; gi <= RZ; gi += 3) {
            step(A, Bp, C, gi);
            if (gi + 1 > RZ) break;
            step(Bp, C, A, gi + 1);
            if (gi + 2 > RZ) break;
            step(C, A, Bp, gi + 2);
        }
        if (sl >= 1) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&done[q & 1]);
        }
    }
    if (t_end == nt) {
        // base slice nt-1 has no later slice: its cubes use that slice alone
        const int q = nslab - 1;
        uint32_t *bq = bm + (q & 1) * RZ * L.rw;
        if (ok && q >= 2 && !wait_ab(&freed[q & 1], ((q >> 1) - 1) & 1, abort)) ok = false;
        ok = __all_sync(ALL, ok);
        if (ok) {
            for (int ci = 0; ci < ncz; ++ci) {
                int nsv = 0;
#pragma unroll
                for (int r = 0; r < S3_RPW; ++r) {
                    const int cr = gr0 + r;
                    if (cr >= ncy) break;
                    const uint32_t P = TS[((ci * RY + cr) * XC + c) * 32 + lane];
                    const uint32_t mixed = (P >> 16) & ~P & 0xFFFu;
                    const uint32_t sv = mixed & (mixed >> 4) & (mixed >> 8) & gmask;
                    if (sv) {
                        const int idx = cr * nx + xb;
                        atomicOr(&bq[ci * L.rw + (idx >> 5)], sv << (idx & 31));
                        nsv += __popc(sv);
                    }
                }
                nsv = __reduce_add_sync(ALL, nsv);
                if (lane == 0 && nsv) atomicAdd(&scnt[(q & 1) * RZ + ci], nsv);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&done[q & 1]);
    }
    if (!ok) atomicOr(status, ST_TIMEOUT);
    if (!EXACT) bad |= ((qa_and ^ MAGIC_BITS) | (qa_or ^ MAGIC_BITS)) & 0xFF800000u;
    if (bad) atomicOr(status, EXACT ? ST_RANGE : ST_WIDE);
}

template <bool EXACT>
void *s3_kernel(int nx) {
    const int xc = s3_chunks(nx);
    if (xc == 1) return (void *)k_detect3_stream<EXACT, 1>;
    if (xc == 2) return (void *)k_detect3_stream<EXACT, 2>;
    if (xc == 4) return (void *)k_detect3_stream<EXACT, 4>;
    return (void *)k_detect3_stream<EXACT, 8>;
}

}  // namespace

// ---- host side: launch configuration ----
size_t stream3_smem_bytes(int nx, const Blocking &B) { return (size_t)s3_layout(nx, B.ry, B.rz).total; }
int stream3_threads(int nx) { return s3_threads(nx); }
int stream3_ry(int nx) { return s3_grows(nx) - 1; }

int stream3_ctas_per_sm(int nx, const Blocking &B) {
    int n = 0;
    const size_t smem = stream3_smem_bytes(nx, B);
    const void *k = s3_kernel<false>(nx);
    raise_smem_cap(k, smem, false);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, s3_threads(nx), smem);
    return n > 0 ? n : 1;
}

cudaError_t launch_detect3(int variant, const Field &F, const Blocking &B, const Workspace &W, cudaStream_t s,
                           bool capturing) {
    // the consumer warps read rows y0-1 .. y0+ry+1 of each plane chunk: the
    // unit's cube rows must be the warps' G rows less one
    if (B.ry != stream3_ry(F.pitch) || F.pitch % 4 != 0 || F.pitch > STREAM3_MAX_NX) return cudaErrorInvalidValue;
    const bool exact = variant == VAR_STREAM3_EXACT;
    const void *k = exact ? s3_kernel<true>(F.pitch) : s3_kernel<false>(F.pitch);
    const size_t smem = stream3_smem_bytes(F.pitch, B);
    // the cap only ever grows: a captured graph may replay a larger launch
    // after a smaller one was configured
    const cudaError_t e = raise_smem_cap(k, smem, capturing);
    if (e != cudaSuccess) return e;
    const unsigned units = (unsigned)((long long)B.ntc * B.nzb * B.nyb);
    Field Fa = F;
    Blocking Ba = B;
    Workspace Wa = W;
    void *args[] = {&Fa, &Ba, &Wa};
    return cudaLaunchKernel(k, dim3(units), dim3(s3_threads(F.pitch)), args, smem, s);
}

}  // namespace ftk
