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
//  * consumer warps: per G plane z (z0 .. z0+rz) each warp takes a run of
//    G rows of one 128-column chunk; a lane quantises 4 consecutive samples
//    (F = rint(f 2^S) in a magic-number encoding, exact for |F| <= 2^22;
//    wider values flag an exact re-run), takes the central differences in x,
//    y and z and packs the 12 sign bits (G_r < 0; zero counts as positive)
//    into one word, kept twice (an AND half and an OR half).  After a named
//    barrier the warps combine, per cube row, the words of the cube's 8
//    spatial corners (rows y, y+1; planes z, z+1; columns x, x+1) and then
//    the words of the two slices t, t+1 (the previous slice's cube words
//    stay in smem).  A cube survives iff every gradient component has
//    corners of both signs; that test is exact, because the symbolic
//    perturbation is infinitesimal and adds a positive term to a zero
//    component.  Survivors go to a double-buffered smem bitmap;
//  * compactor warp: per base slice, turns the bitmap into ordered lists of
//    surviving cubes, one per segment (t, z, y-block), in global memory.
// Grid edges need no special cases in the sign code: clamped rows, planes
// and columns turn every one-sided difference into a doubled central
// difference of the same sign, and a cube whose upper corners leave the grid
// repeats its lower corners (the faces it owns then lie in the grid's
// boundary).  Every wait is bounded; a wait that runs out sets a shared abort
// flag, every warp drains and the run reports ST_TIMEOUT.
#include <cuda_runtime.h>

#include <climits>

#include "ftk_kernels.cuh"
#include "ftk_tma.cuh"

namespace ftk {

namespace {

constexpr int S3_NW = 4;                  // consumer warps (each takes 4 of 16 G rows per plane)
constexpr int S3_NS = 5;                  // smem ring slots (plane chunks)
constexpr int S3_THREADS = (S3_NW + 2) * 32;
constexpr float S3_RANGE = 268435456.0f;  // 2^28
constexpr uint32_t ALL = 0xffffffffu;

__host__ __device__ inline int s3_round16(int v) { return (v + 15) & ~15; }
// 128-column chunks per row (a power of two, so that the warps split evenly)
__host__ __device__ inline int s3_chunks(int nx) { return nx <= 128 ? 1 : nx <= 256 ? 2 : 4; }

struct S3Layout {
    int slot_floats, ring, bars, abort, sr, ts, bm, rw, cnt, total;
};
__host__ __device__ inline S3Layout s3_layout(int nx, int ry, int rz) {
    constexpr int ns = S3_NS;
    S3Layout L;
    const int xc = s3_chunks(nx);
    L.slot_floats = (ry + 3) * nx;                 // nx % 4 == 0: a multiple of 16 bytes
    L.ring = 0;
    L.bars = L.ring + ns * L.slot_floats * 4;
    L.abort = L.bars + (2 * ns + 4) * 8;
    L.sr = s3_round16(L.abort + 4);
    L.ts = L.sr + 3 * (ry + 1) * xc * 32 * 4;      // sign words of 3 G planes
    L.bm = L.ts + rz * ry * xc * 32 * 4;           // cube words of the previous slice
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

template <bool EXACT>
__global__ void __launch_bounds__(S3_THREADS, 3) k_detect3_stream(Field F, Blocking B, Workspace W) {
    extern __shared__ __align__(128) unsigned char smem[];
    // the sweep covers the padded row (pitch columns, the padding repeating
    // column nx-1); survivors are the grid's (columns < nxl)
    const int nx = F.pitch, nxl = F.nx, ny = F.ny, nz = F.nz, nt = F.nt;
    const int RY = B.ry, RZ = B.rz;
    constexpr int NS = S3_NS;
    const int XC = s3_chunks(nx);
    const S3Layout L = s3_layout(nx, RY, RZ);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *ring = reinterpret_cast<float *>(smem + L.ring);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint64_t *empty = full + NS;
    uint64_t *done = empty + NS;     // [2] slab bits complete (consumer warps arrive)
    uint64_t *freed = done + 2;      // [2] bitmap compacted and cleared (compactor arrives)
    volatile int *abort = reinterpret_cast<volatile int *>(smem + L.abort);
    uint32_t *SR = reinterpret_cast<uint32_t *>(smem + L.sr);
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
    const int GR = RY + 1;                // G rows per plane

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
        // words are dealt to the lanes round-robin (dense regions spread over
        // the warp); pass 1 counts, pass 2 writes in bitmap order
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
    const int NG = S3_NW / XC;             // row groups (warps per chunk)
    const int c = warp % XC;               // this warp's 128-column chunk
    const int grp = warp / XC;
    const int xb = c * 128 + lane * 4;     // first column of this lane
    const bool act = xb < nx;
    const int xa = act ? xb : 0;           // a safe address for idle lanes
    const bool xlast = act && xb + 4 >= nx;
    // the lane's columns inside the grid (the rest is padding)
    const uint32_t gmask = act ? (1u << max(0, min(4, nxl - xb))) - 1u : 0u;
    const int gper = (GR + NG - 1) / NG;
    const int gr0 = min(GR, grp * gper), gr1 = min(GR, gr0 + gper);
    const int cper = (RY + NG - 1) / NG;
    const int cr0 = min(RY, grp * cper), cr1 = min(RY, cr0 + cper);
    const float scale = F.scale;
    uint32_t bad = 0, qa_and = 0xffffffffu, qa_or = 0u;
    bool any = false;
    bool ok = true;

    auto srw = [&](int buf, int row, int cc) -> uint32_t * { return SR + ((buf * GR + row) * XC + cc) * 32; };
    // offset (floats) of this lane's first column of grid row yy (clamped)
    // within a plane chunk
    auto roff = [&](int yy) -> int { return (min(max(yy, 0), ny - 1) - ylo) * nx + xa; };
    const int yfirst = y0 + gr0;
    const int ngr = max(0, min(gr1, ny - y0) - gr0);       // this warp's G rows inside the grid
    // halo sample of this lane: lane 0 the column left of the chunk (itself
    // at x = 0), lane 31 the column right of it (unused at the grid's edge)
    const int hoff = !act ? 0 : lane == 0 ? (xa == 0 ? 0 : -1) : (lane == 31 && !xlast ? 4 : 0);
    // cube word of chunk cc, lane l of cube row (rows cr, cr2) between G planes a and b
    auto cube_word = [&](int ba, int bb, int cr, int cr2, int cc, int l) -> uint32_t {
        const uint32_t t0w = cmb(srw(ba, cr, cc)[l], srw(bb, cr, cc)[l]);
        const uint32_t t1w = cmb(srw(ba, cr2, cc)[l], srw(bb, cr2, cc)[l]);
        return cmb(t0w, t1w);
    };
    // the lane's 4 cubes are 4 consecutive bits of one word (idx % 4 == 0)
    auto emit = [&](uint32_t *bq, int ci, int cr, uint32_t sv) {
        const int idx = cr * nx + xb;
        atomicOr(&bq[ci * L.rw + (idx >> 5)], sv << (idx & 31));
    };
    // adds the warp's survivors of cube plane ci (this lane: n) to its count
    auto count = [&](int buf, int ci, int n) {
        n = __reduce_add_sync(ALL, n);
        if (lane == 0 && n) atomicAdd(&scnt[buf * RZ + ci], n);
    };

    for (int sl = 0; sl < nsl; ++sl) {
        const int q = sl - 1;              // slab completed by this slice
        const int jb = sl * PL;
        uint32_t *bq = bm + (q & 1) * RZ * L.rw;
        if (ok && q >= 2 && !wait_ab(&freed[q & 1], ((q >> 1) - 1) & 1, abort)) ok = false;
        ok = __all_sync(ALL, ok);
        for (int gi = 0; gi <= RZ; ++gi) {
            // the three plane chunks of G plane gi: loads jb+gi .. jb+gi+2
            for (int jj = gi == 0 ? jb : jb + gi + 2; jj <= jb + gi + 2; ++jj)
                if (ok && !wait_ab(&full[jj % NS], (jj / NS) & 1, abort)) ok = false;
            ok = __all_sync(ALL, ok);
            if (ok && z0 + gi <= nz - 1 && ngr > 0) {
                const float *pm = ring + (size_t)((jb + gi) % NS) * L.slot_floats;
                const float *p0 = ring + (size_t)((jb + gi + 1) % NS) * L.slot_floats;
                const float *pp = ring + (size_t)((jb + gi + 2) % NS) * L.slot_floats;
                uint32_t *dst = SR + (((gi % 3) * GR + gr0) * XC + c) * 32 + lane;
                // rolling rows y-1 (a), y (b) of the own plane, quantised, and
                // the lane's halo sample of row y
                const int ob0 = roff(yfirst);
                const float4 va = *reinterpret_cast<const float4 *>(p0 + roff(yfirst - 1));
                const float4 vb = *reinterpret_cast<const float4 *>(p0 + ob0);
                uint32_t a0 = q3<EXACT>(va.x, scale, bad), a1 = q3<EXACT>(va.y, scale, bad);
                uint32_t a2 = q3<EXACT>(va.z, scale, bad), a3 = q3<EXACT>(va.w, scale, bad);
                uint32_t b0 = q3<EXACT>(vb.x, scale, bad), b1 = q3<EXACT>(vb.y, scale, bad);
                uint32_t b2 = q3<EXACT>(vb.z, scale, bad), b3 = q3<EXACT>(vb.w, scale, bad);
                uint32_t hb = q3<EXACT>(p0[ob0 + hoff], scale, bad);
#pragma unroll 2
                for (int r = 0; r < ngr; ++r) {
                    const int y = yfirst + r;
                    const int o0 = roff(y), oc = roff(y + 1);
                    const float4 vc = *reinterpret_cast<const float4 *>(p0 + oc);
                    const float4 vm = *reinterpret_cast<const float4 *>(pm + o0);
                    const float4 vp = *reinterpret_cast<const float4 *>(pp + o0);
                    const uint32_t hc = q3<EXACT>(p0[oc + hoff], scale, bad);
                    const uint32_t c0 = q3<EXACT>(vc.x, scale, bad), c1 = q3<EXACT>(vc.y, scale, bad);
                    const uint32_t c2 = q3<EXACT>(vc.z, scale, bad), c3 = q3<EXACT>(vc.w, scale, bad);
                    const uint32_t m0 = q3<EXACT>(vm.x, scale, bad), m1 = q3<EXACT>(vm.y, scale, bad);
                    const uint32_t m2 = q3<EXACT>(vm.z, scale, bad), m3 = q3<EXACT>(vm.w, scale, bad);
                    const uint32_t p0q = q3<EXACT>(vp.x, scale, bad), p1q = q3<EXACT>(vp.y, scale, bad);
                    const uint32_t p2q = q3<EXACT>(vp.z, scale, bad), p3q = q3<EXACT>(vp.w, scale, bad);
                    // columns xb-1 and xb+4 (clamped) of the own row: neighbours'
                    // samples, or this lane's halo sample at the warp's edges
                    const uint32_t up = __shfl_up_sync(ALL, b3, 1);
                    const uint32_t dn = __shfl_down_sync(ALL, b0, 1);
                    const uint32_t lq = lane == 0 ? hb : up;
                    const uint32_t rq = xlast ? b3 : lane == 31 ? hb : dn;
                    if (!EXACT && act) {
                        // own samples must lie in the fast encoding's range (the
                        // exact form checks every sample it quantises)
                        qa_and &= b0 & b1 & b2 & b3;
                        qa_or |= b0 | b1 | b2 | b3;
                        any = true;
                    }
                    uint32_t w = 0;
                    w = __funnelshift_l(qd<EXACT>(p3q, m3), w, 1);
                    w = __funnelshift_l(qd<EXACT>(p2q, m2), w, 1);
                    w = __funnelshift_l(qd<EXACT>(p1q, m1), w, 1);
                    w = __funnelshift_l(qd<EXACT>(p0q, m0), w, 1);
                    w = __funnelshift_l(qd<EXACT>(c3, a3), w, 1);
                    w = __funnelshift_l(qd<EXACT>(c2, a2), w, 1);
                    w = __funnelshift_l(qd<EXACT>(c1, a1), w, 1);
                    w = __funnelshift_l(qd<EXACT>(c0, a0), w, 1);
                    w = __funnelshift_l(qd<EXACT>(rq, b2), w, 1);
                    w = __funnelshift_l(qd<EXACT>(b3, b1), w, 1);
                    w = __funnelshift_l(qd<EXACT>(b2, b0), w, 1);
                    w = __funnelshift_l(qd<EXACT>(b1, lq), w, 1);
                    dst[r * XC * 32] = w | (w << 16);
                    a0 = b0; a1 = b1; a2 = b2; a3 = b3;
                    b0 = c0; b1 = c1; b2 = c2; b3 = c3;
                    hb = hc;
                }
            }
            // release the plane chunk that no later G plane of this slice reads
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[(jb + gi) % NS]);
                if (gi == RZ) {
                    mbar_arrive(&empty[(jb + RZ + 1) % NS]);
                    mbar_arrive(&empty[(jb + RZ + 2) % NS]);
                }
            }
            named_sync(1, S3_NW * 32);
            const int ci = gi - 1;             // cube plane between G planes gi-1 and gi
            if (ok && gi >= 1 && ci < ncz) {
                const int ba = ci % 3;
                const int bb = z0 + ci + 1 <= nz - 1 ? gi % 3 : ba;
                const int rs = XC * 32;               // SR / TS row stride (words)
                const uint32_t *pa = SR + ((ba * GR + cr0) * XC + c) * 32 + lane;
                const uint32_t *pb = SR + ((bb * GR + cr0) * XC + c) * 32 + lane;
                uint32_t *ts = TS + ((ci * RY + cr0) * XC + c) * 32 + lane;
                uint32_t top = cr0 < ncy ? cmb(pa[0], pb[0]) : 0u;
                int nsv = 0;
                for (int cr = cr0; cr < cr1; ++cr) {
                    if (cr >= ncy) break;
                    const bool step = y0 + cr + 1 <= ny - 1;   // else the cube repeats row ny-1
                    const uint32_t bot = step ? cmb(pa[rs], pb[rs]) : top;
                    const uint32_t u = cmb(top, bot);
                    // the cube's x+1 corners: the next lane's first column
                    uint32_t nxt = __shfl_down_sync(ALL, u, 1);
                    if (lane == 31 && c + 1 < XC) {
                        const int cr2 = step ? cr + 1 : cr;
                        nxt = cube_word(ba, bb, cr, cr2, c + 1, 0);
                    }
                    uint32_t nb = ((u >> 1) & 0x07770777u) | ((nxt & 0x01110111u) << 3);
                    if (xlast) nb = (nb & ~0x08880888u) | (u & 0x08880888u);   // column nx-1
                    const uint32_t P = cmb(u, nb);
                    if (sl >= 1 && act) {
                        const uint32_t c4 = cmb(P, *ts);
                        const uint32_t mixed = (c4 >> 16) & ~c4 & 0xFFFu;
                        const uint32_t sv = mixed & (mixed >> 4) & (mixed >> 8) & gmask;
                        if (sv) {
                            emit(bq, ci, cr, sv);
                            nsv += __popc(sv);
                        }
                    }
                    *ts = P;
                    ts += rs;
                    pa += rs;
                    pb += rs;
                    top = bot;
                }
                if (sl >= 1) count(q & 1, ci, nsv);
            }
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
                for (int cr = cr0; cr < cr1 && cr < ncy; ++cr) {
                    const uint32_t P = TS[((ci * RY + cr) * XC + c) * 32 + lane];
                    const uint32_t mixed = (P >> 16) & ~P & 0xFFFu;
                    const uint32_t sv = mixed & (mixed >> 4) & (mixed >> 8) & gmask;
                    if (sv) {
                        emit(bq, ci, cr, sv);
                        nsv += __popc(sv);
                    }
                }
                count(q & 1, ci, nsv);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&done[q & 1]);
        }
    }
    if (!ok) atomicOr(status, ST_TIMEOUT);
    if (!EXACT && any) bad |= ((qa_and ^ MAGIC_BITS) | (qa_or ^ MAGIC_BITS)) & 0xFF800000u;
    if (bad) atomicOr(status, EXACT ? ST_RANGE : ST_WIDE);
}

template <bool EXACT>
void *s3_kernel() { return (void *)k_detect3_stream<EXACT>; }

}  // namespace

// ---- host side: launch configuration ----
size_t stream3_smem_bytes(int nx, const Blocking &B) { return (size_t)s3_layout(nx, B.ry, B.rz).total; }
int stream3_threads() { return S3_THREADS; }

int stream3_ctas_per_sm(int nx, const Blocking &B) {
    int n = 0;
    const size_t smem = stream3_smem_bytes(nx, B);
    const void *k = s3_kernel<false>();
    raise_smem_cap(k, smem, false);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, S3_THREADS, smem);
    return n > 0 ? n : 1;
}

cudaError_t launch_detect3(int variant, const Field &F, const Blocking &B, const Workspace &W, cudaStream_t s,
                           bool capturing) {
    const bool exact = variant == VAR_STREAM3_EXACT;
    const void *k = exact ? s3_kernel<true>() : s3_kernel<false>();
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
    return cudaLaunchKernel(k, dim3(units), dim3(S3_THREADS), args, smem, s);
}

}  // namespace ftk
