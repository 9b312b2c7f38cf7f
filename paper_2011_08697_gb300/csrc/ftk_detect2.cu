// Streaming sign cull for 2D fields (2D + time, paper Sec. 3.3 mesh, Sec. 4.1
// predicate): the dense, HBM-bound pass of the 2D pipeline.  The sparse
// stages that follow it are in ftk_kernels.cu.
#include <cuda_runtime.h>

#include <climits>

#include "ftk_kernels.cuh"
#include "ftk_tma.cuh"

namespace ftk {

__host__ __device__ inline int s2_round16(int v) { return (v + 15) & ~15; }

// ----------------------------------------------------------------------------
// Streaming 2D detect kernel (rows of nx % 4 == 0 floats, 16-byte aligned).
//
// One CTA per unit = (block of RY2 cube rows, time chunk), three warp roles:
//  * producer warp: streams the unit's rows -- slice after slice, the clamped
//    rows y0-1 .. y0+RY2+1 -- into a ring of NS2 shared-memory row slots with
//    1D bulk TMA copies (cp.async.bulk; an mbarrier per slot counts the
//    bytes, a second one counts the consumer warps that released the slot);
//  * consumer warps: a thread owns CX = 8 columns; it reads each row once
//    (two float4 plus three clamped neighbours), quantises, forms the integer
//    gradient of the previous row and packs the 18 sign bits of (G_x, G_y) at
//    9 columns with funnel shifts.  The exact cube cull of its 8 cubes is
//    then bit-parallel: AND/OR of x pairs, y pairs (previous row) and time
//    pairs (one 32-bit word per cube row kept in a register across slices).
//    Grid edges need no branches in the row code: clamped rows/columns make
//    every one-sided difference a doubled central difference;
//  * compactor warp: at the end of each slab it turns the slab's survivor
//    bitmap (double-buffered; mbarrier handshake with the consumers) into an
//    ordered list of surviving cubes in global memory.
// No CTA-wide barrier runs inside the main loop.
// ----------------------------------------------------------------------------
constexpr int RY2 = STREAM2_ROWS;   // cube rows per unit
constexpr int NS2 = 8;        // TMA ring slots (rows)
constexpr int CX = 8;         // columns per consumer thread
// quantised sample in offset encoding: MAGIC_BITS + rint(v 2^S) (mod 2^32);
// differences of two encodings are exact integer differences
template <bool EXACT>
__device__ __forceinline__ uint32_t qbits(float v, float scale, uint32_t &bad) {
    if (EXACT) {
        const float w = v * scale;
        if (!(fabsf(w) <= RANGE_LIMIT)) bad |= 1u;
        return (uint32_t)(fabsf(w) <= RANGE_LIMIT ? __float2int_rn(w) : 0) + MAGIC_BITS;
    }
    // v * 2^S + 1.5 * 2^23 rounds to the nearest integer (ties to even) in
    // the mantissa whenever |v * 2^S| <= 2^22; bits - MAGIC_BITS = rint(v 2^S)
    return __float_as_uint(__fmaf_rn(v, scale, MAGIC_F));
}

__host__ __device__ inline int stream2_consumers(int nx) { return ((nx + CX - 1) / CX + 31) / 32 * 32; }

struct Stream2Layout {
    int ring, bars, bm, bmw, cnt, st, total;
};
// comps = 2: a ring slot holds a row of vectors (two floats per vertex)
__host__ __device__ inline Stream2Layout stream2_layout(int nx, int comps = 1) {
    Stream2Layout L;
    L.ring = 0;
    L.bars = L.ring + NS2 * nx * comps * 4;
    L.bmw = (RY2 * nx + 31) / 32;
    L.bm = s2_round16(L.bars + (2 * NS2 + 4) * 8);
    L.cnt = L.bm + 2 * L.bmw * 4;     // [2] survivors per slab buffer
    L.st = s2_round16(L.cnt + 2 * 4); // [RY2][consumers] cube-row words of the previous slice
    L.total = s2_round16(L.st + RY2 * stream2_consumers(nx) * 4);
    return L;
}

// Word of one G row's pairs: bits 0-7 / 16-23 = G_x / G_y "both corners of the
// x pair negative" (AND), bits 8-15 / 24-31 = "some corner negative" (OR).
// Input: sign bits of G_x at bits 0-8 and of G_y at bits 16-24.
__device__ __forceinline__ uint32_t pair_word(uint32_t w) {
    const uint32_t s = w >> 1;
    return ((w & s) & 0x00FF00FFu) | (((w | s) & 0x00FF00FFu) << 8);
}
// AND on the all-negative bits, OR on the some-negative bits
__device__ __forceinline__ uint32_t combine(uint32_t a, uint32_t b) {
    return ((a & b) & 0x00FF00FFu) | ((a | b) & 0xFF00FF00u);
}
// cubes (bit k) where both components have corners of both signs
__device__ __forceinline__ uint32_t survivors8(uint32_t c) {
    const uint32_t mixed = (c >> 8) & ~c & 0x00FF00FFu;
    return mixed & (mixed >> 16) & 0xFFu;
}

// VEC: a 2D vector field (two components per vertex, interleaved): the
// vectors themselves take the gradients' place, so a slice streams only the
// unit's rows y0 .. y0+RY2 and a G row is the row itself
template <bool EXACT, int MAXT, int MINB, bool VEC = false>
__global__ void __launch_bounds__(MAXT, MINB) k_detect2_stream(Field F, Blocking B, Workspace W) {
    extern __shared__ __align__(128) unsigned char smem[];
    // the sweep covers the padded row (pitch columns; padding repeats column
    // nx-1, so every grid vertex's gradient signs are exact and the extra
    // corners only make cubes survive more easily); survivors are the grid's
    const int nx = F.pitch, nxl = F.nx, ny = F.ny, nt = F.nt;
    const int NC = (int)blockDim.x - 64;
    const int CW = NC >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int CMP = VEC ? 2 : 1;        // floats per vertex
    const Stream2Layout L = stream2_layout(nx, CMP);
    float *ring = reinterpret_cast<float *>(smem + L.ring);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint64_t *empty = full + NS2;
    uint64_t *done = empty + NS2;    // [2] slab bits complete (consumer warps arrive)
    uint64_t *freed = done + 2;      // [2] bitmap compacted and cleared (compactor arrives)
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem + L.bm);   // [2][bmw]
    int *scnt = reinterpret_cast<int *>(smem + L.cnt);          // [2]
    unsigned *status = &W.ctr->status;

    const int tci = blockIdx.x % B.ntc;
    const int yb = blockIdx.x / B.ntc;
    const int y0 = yb * RY2;
    const int t0 = tci * B.tc;
    const int t_end = min(nt, t0 + B.tc);
    const int s_last = min(t_end, nt - 1);
    const int nsl = s_last - t0 + 1;      // slices of the unit
    const int nslab = t_end - t0;         // slabs (base slices) owned
    constexpr int RS = VEC ? RY2 + 1 : RY2 + 3;   // rows streamed per slice
    const int sl0 = B.st_mode == 2 ? 1 : 0;   // slice 0's words come from st_in
    const int J = (nsl - sl0) * RS;

    if (threadIdx.x == 0) {
        for (int k = 0; k < NS2; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], CW);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&done[b], CW);
            mbar_init(&freed[b], 1);
        }
        mbar_fence_init();
    }
    for (int i = threadIdx.x; i < 2 * L.bmw; i += blockDim.x) bm[i] = 0u;
    if (threadIdx.x < 2) scnt[threadIdx.x] = 0;
    __syncthreads();

    if (warp == CW) {
        // ---------------- producer ----------------------------------------
        if (lane == 0) {
            int issued = 0;
            bool ok = true;
            for (int j = 0; j < J; ++j) {
                const int slot = j % NS2;
                if (j >= NS2 && !mbar_wait(&empty[slot], ((j / NS2) + 1) & 1, 64)) {
                    ok = false;
                    break;
                }
                const int s = t0 + sl0 + j / RS;
                const int y = min(max((VEC ? y0 : y0 - 1) + j % RS, 0), ny - 1);
                const uint32_t bytes = (uint32_t)nx * CMP * 4u;
                mbar_arrive_expect_tx(&full[slot], bytes);
                tma_row(ring + (size_t)slot * nx * CMP, F.f + ((long long)s * ny + y) * nx * CMP, bytes, &full[slot]);
                issued = j + 1;
            }
            if (!ok) {
                atomicOr(status, ST_TIMEOUT);
                // never leave a copy in flight into a CTA that is exiting
                for (int j = max(0, issued - NS2); j < issued; ++j) mbar_wait(&full[j % NS2], (j / NS2) & 1);
            }
        }
        return;
    }
    if (warp == CW + 1) {
        // ---------------- compactor ---------------------------------------
        // words are dealt to the lanes round-robin (dense regions spread over
        // the warp); pass 1 counts, pass 2 writes in bitmap order
        for (int q = 0; q < nslab; ++q) {
            const int b = q & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&done[b], (q >> 1) & 1, 256))) {
                if (lane == 0) atomicOr(status, ST_TIMEOUT);
                return;
            }
            const int total = scnt[b];
            const int t = t0 + q;
            const long long seg = (long long)t * B.nyb + yb;
            long long base = 0;
            if (lane == 0) {
                base = total ? (long long)atomicAdd(&W.ctr->survivors, (unsigned long long)total) : 0;
                W.seg_scnt[seg] = total;
                W.seg_sstage[seg] = base;
                if (base + total > W.scap) atomicOr(status, ST_SOVERFLOW);
            }
            if (total > 0) {
                base = __shfl_sync(0xffffffffu, base, 0);
                compact_bits<16>(bm + b * L.bmw, L.bmw, nx, nxl, 1.0f / (float)nx, (long long)t * ny + y0, base,
                                 W.surv, W.scap);
            }
            __syncwarp();
            if (lane == 0) scnt[b] = 0;
            __syncwarp();
            if (lane == 0) mbar_arrive(&freed[b]);
        }
        return;
    }

    // ---------------- consumers ---------------------------------------------
    const int x0 = (int)threadIdx.x * CX;
    const bool act = x0 < nx;
    const int ncol = act ? min(CX, nx - x0) : 0;           // 8, or 4 on the last thread
    const int ngrid = act ? max(0, min(CX, nxl - x0)) : 0;       // columns inside the grid
    const uint32_t vmask = (ncol == 8 ? 0xFFu : ncol == 4 ? 0x0Fu : 0u) & ((1u << ngrid) - 1u);
    const int xa = act ? x0 : 0;                           // safe address for idle threads
    const int xb = ncol == 8 ? x0 + 4 : xa;                // second float4 (duplicate when absent)
    const int xl = max(xa - 1, 0);
    const int xr1 = min(xa + CX, nx - 1);
    const int xr2 = min(xa + CX + 1, nx - 1);
    const bool dbl7 = ncol == 8 && x0 + 8 == nx;           // column 7 is x = nx-1
    const bool dbl3 = ncol == 4;                           // column 3 is x = nx-1
    const float scale = F.scale;
    uint32_t bad = 0, dummy = 0;
    // cube-row words of the previous slice, one smem column per thread
    // (row i at sst[i * NC]): indexed by the row, so the row loop need not be
    // unrolled completely
    uint32_t *sst = reinterpret_cast<uint32_t *>(smem + L.st) + threadIdx.x;
    for (int i = 0; i < RY2; ++i) sst[i * NC] = 0;
    // incremental mode: slice 0's cube-row words from the previous push
    const long long st_base = ((long long)yb * RY2) * NC + threadIdx.x;
    if (B.st_mode == 2) {
#pragma unroll
        for (int i = 0; i < RY2; ++i) sst[i * NC] = B.st_in[st_base + (long long)i * NC];
    }
    uint32_t fa[11], fb[11], fc[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) fa[k] = fb[k] = fc[k] = MAGIC_BITS;
    uint32_t pprev = 0;
    // fast encoding: AND and OR of every sample read, checked against the
    // encoding's range once at the end
    uint32_t qa_and = 0xffffffffu, qa_or = 0u;
    int j = 0;
    int nsv = 0;     // survivors this thread found in the current slab
    bool ok = true;

    // Streamed row vi of slice sl: wait for its ring slot, quantise it into
    // `cur`, and with the two rows before it (r0 = row u-1, r1 = row u) form
    // G row u = y0 - 2 + vi and the cube rows it completes.  The caller
    // rotates the three row buffers through the arguments, so no row is
    // copied.  Only the signs of G matter here: the one-sided difference at
    // a grid edge (clamped rows and columns) has the sign of the doubled
    // difference the exact stages use.
    auto row = [&](int vi, int sl, uint32_t *bq, const uint32_t (&r0)[11], const uint32_t (&r1)[11],
                   uint32_t (&cur)[11]) {
        const int slot = j % NS2;
        if (ok && !mbar_wait(&full[slot], (j / NS2) & 1)) ok = false;
        ok = __all_sync(0xffffffffu, ok);   // keep the warp converged
        if (ok) {
            const float *r = ring + (size_t)slot * nx;
            const float4 c0 = *reinterpret_cast<const float4 *>(r + xa);
            const float4 c1 = *reinterpret_cast<const float4 *>(r + xb);
            cur[1] = qbits<EXACT>(c0.x, scale, bad);
            cur[2] = qbits<EXACT>(c0.y, scale, bad);
            cur[3] = qbits<EXACT>(c0.z, scale, bad);
            cur[4] = qbits<EXACT>(c0.w, scale, bad);
            cur[5] = qbits<EXACT>(c1.x, scale, bad);
            cur[6] = qbits<EXACT>(c1.y, scale, bad);
            cur[7] = qbits<EXACT>(c1.z, scale, bad);
            cur[8] = qbits<EXACT>(c1.w, scale, bad);
            if (ncol == 4) {
                // columns x0+4.. do not exist: clamp to column nx-1
                cur[5] = cur[6] = cur[7] = cur[8] = cur[4];
            }
            cur[0] = qbits<EXACT>(r[xl], scale, dummy);
            cur[9] = qbits<EXACT>(r[xr1], scale, dummy);
            cur[10] = qbits<EXACT>(r[xr2], scale, dummy);
            if (!EXACT) {
                // every sample read is a sample of the field (idle threads
                // read column 0): all must lie in the fast rounding range
                qa_and &= cur[1] & cur[2] & cur[3] & cur[4] & cur[5] & cur[6] & cur[7] & cur[8];
                qa_or |= cur[1] | cur[2] | cur[3] | cur[4] | cur[5] | cur[6] | cur[7] | cur[8];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
        ++j;
        const int u = y0 - 2 + vi;
        if (vi >= 2 && u <= ny - 1) {
            uint32_t gx[9], gy[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                gx[k] = r1[k + 2] - r1[k];
                gy[k] = cur[k + 1] - r0[k + 1];
            }
            if (dbl7) { gx[8] = gx[7]; gy[8] = gy[7]; }      // no column x0+8: duplicate
            if (dbl3) { gx[4] = gx[3]; gy[4] = gy[3]; }      // no column x0+4
            // bit 31 of each (wrapped) difference is the sign of G:
            // w = sign(G_x[k]) at bit k, sign(G_y[k]) at bit 16 + k
            uint32_t w = 0;
#pragma unroll
            for (int k = 8; k >= 0; --k) w = __funnelshift_l(gy[k], w, 1);
            w <<= 7;
#pragma unroll
            for (int k = 8; k >= 0; --k) w = __funnelshift_l(gx[k], w, 1);
            const uint32_t p = pair_word(w);
            // cube row c = u-1 (G rows u-1, u); at the top edge cube row u alone
            if (vi >= 3) {
                const int i = vi - 3;
                const uint32_t sq = combine(pprev, p);
                if (sl > 0) {
                    const uint32_t sv8 = survivors8(combine(sq, sst[i * NC])) & vmask;
                    if (sv8) {
                        const int idx = i * nx + x0;
                        atomicOr(&bq[idx >> 5], sv8 << (idx & 31));
                        nsv += __popc(sv8);
                        if ((idx & 31) > 24) atomicOr(&bq[(idx >> 5) + 1], sv8 >> (32 - (idx & 31)));
                    }
                }
                sst[i * NC] = sq;
            }
            if (u == ny - 1 && vi - 2 < RY2) {
                const int i = vi - 2;
                if (sl > 0) {
                    const uint32_t sv8 = survivors8(combine(p, sst[i * NC])) & vmask;
                    if (sv8) {
                        const int idx = i * nx + x0;
                        atomicOr(&bq[idx >> 5], sv8 << (idx & 31));
                        nsv += __popc(sv8);
                        if ((idx & 31) > 24) atomicOr(&bq[(idx >> 5) + 1], sv8 >> (32 - (idx & 31)));
                    }
                }
                sst[i * NC] = p;
            }
            pprev = p;
        }
    };

    // Vector rows: streamed row vi of slice sl is G row u = y0 + vi; the
    // sign of a quantised component is bit 31 of its encoding minus the
    // encoding of zero.  Cube row u-1 completes with G rows u-1 and u; at
    // the top edge cube row u uses row u alone.
    auto row_vec = [&](int vi, int sl, uint32_t *bq) {
        const int slot = j % NS2;
        uint32_t w = 0;
        if (ok && !mbar_wait(&full[slot], (j / NS2) & 1)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
            const float *r = ring + (size_t)slot * nx * 2;
            float v[18];
            const float4 c0 = *reinterpret_cast<const float4 *>(r + 2 * xa);
            const float4 c1 = *reinterpret_cast<const float4 *>(r + 2 * xa + 4);
            const float4 c2 = *reinterpret_cast<const float4 *>(r + 2 * xb);
            const float4 c3 = *reinterpret_cast<const float4 *>(r + 2 * xb + 4);
            const float2 c4 = *reinterpret_cast<const float2 *>(r + 2 * xr1);
            v[0] = c0.x; v[1] = c0.y; v[2] = c0.z; v[3] = c0.w;
            v[4] = c1.x; v[5] = c1.y; v[6] = c1.z; v[7] = c1.w;
            v[8] = c2.x; v[9] = c2.y; v[10] = c2.z; v[11] = c2.w;
            v[12] = c3.x; v[13] = c3.y; v[14] = c3.z; v[15] = c3.w;
            v[16] = c4.x; v[17] = c4.y;
            uint32_t q[18];
#pragma unroll
            for (int k = 0; k < 18; ++k) q[k] = qbits<EXACT>(v[k], scale, bad);
            if (!EXACT) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    qa_and &= q[k];
                    qa_or |= q[k];
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            // columns: k = 0..7 the thread's, 8 the next (clamped to nx-1);
            // absent columns repeat the last one
            if (ncol == 4) {
#pragma unroll
                for (int k = 8; k < 16; ++k) q[k] = q[k - 2 * (1 + ((k - 8) >> 1))];
            }
#pragma unroll
            for (int k = 8; k >= 0; --k) w = __funnelshift_l(q[2 * k + 1] - MAGIC_BITS, w, 1);
            w <<= 7;
#pragma unroll
            for (int k = 8; k >= 0; --k) w = __funnelshift_l(q[2 * k] - MAGIC_BITS, w, 1);
            if (dbl7) w = (w & ~0x01000100u) | ((w >> 1) & 0x01000100u);   // column x0+8 absent: repeat 7
            if (dbl3) w = (w & ~0x00100010u) | ((w >> 1) & 0x00100010u);   // column x0+4 absent: repeat 3
        }
        ++j;
        const int u = y0 + vi;
        if (u <= ny - 1) {
            const uint32_t p = pair_word(w);
            if (vi >= 1) {
                const int i = vi - 1;
                const uint32_t sq = combine(pprev, p);
                if (sl > 0) {
                    const uint32_t sv8 = survivors8(combine(sq, sst[i * NC])) & vmask;
                    if (sv8) {
                        const int idx = i * nx + x0;
                        atomicOr(&bq[idx >> 5], sv8 << (idx & 31));
                        nsv += __popc(sv8);
                        if ((idx & 31) > 24) atomicOr(&bq[(idx >> 5) + 1], sv8 >> (32 - (idx & 31)));
                    }
                }
                sst[i * NC] = sq;
            }
            if (u == ny - 1 && vi < RY2) {
                const int i = vi;
                if (sl > 0) {
                    const uint32_t sv8 = survivors8(combine(p, sst[i * NC])) & vmask;
                    if (sv8) {
                        const int idx = i * nx + x0;
                        atomicOr(&bq[idx >> 5], sv8 << (idx & 31));
                        nsv += __popc(sv8);
                        if ((idx & 31) > 24) atomicOr(&bq[(idx >> 5) + 1], sv8 >> (32 - (idx & 31)));
                    }
                }
                sst[i * NC] = p;
            }
            pprev = p;
        }
    };

    for (int sl = sl0; sl < nsl && ok; ++sl) {
        // slice sl > 0 completes slab q = sl-1, whose bits go to buffer q & 1:
        // wait until the compactor has released that buffer (slab q-2)
        const int q = sl - 1;
        uint32_t *bq = bm + (q & 1) * L.bmw;
        if (sl > 0 && q >= 2 && !mbar_wait(&freed[q & 1], ((q >> 1) - 1) & 1)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        if constexpr (VEC) {
#pragma unroll 1
            for (int vi = 0; vi < RS; ++vi) row_vec(vi, sl, bq);
        } else {
            // rows in threes, the buffers rotating (fa, fb, fc) -> (fb, fc, fa) -> (fc, fa, fb)
#pragma unroll 1
            for (int vi = 0; vi < RS; vi += 3) {
                row(vi, sl, bq, fa, fb, fc);
                if (vi + 1 < RS) row(vi + 1, sl, bq, fb, fc, fa);
                if (vi + 2 < RS) row(vi + 2, sl, bq, fc, fa, fb);
            }
        }
        if (sl > 0) {
            const int n = __reduce_add_sync(0xffffffffu, nsv);
            if (lane == 0 && n) atomicAdd(&scnt[q & 1], n);
            nsv = 0;
            __syncwarp();
            if (lane == 0) mbar_arrive(&done[q & 1]);
        }
    }
    if (ok && t_end == nt) {
        // base slice nt-1 has no later slice: its cubes use that slice alone
        const int q = nslab - 1;
        uint32_t *bq = bm + (q & 1) * L.bmw;
        if (q >= 2 && !mbar_wait(&freed[q & 1], ((q >> 1) - 1) & 1)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
#pragma unroll
            for (int i = 0; i < RY2; ++i) {
                if (y0 + i < ny) {
                    const uint32_t sv8 = survivors8(sst[i * NC]) & vmask;
                    if (sv8) {
                        const int idx = i * nx + x0;
                        atomicOr(&bq[idx >> 5], sv8 << (idx & 31));
                        nsv += __popc(sv8);
                        if ((idx & 31) > 24) atomicOr(&bq[(idx >> 5) + 1], sv8 >> (32 - (idx & 31)));
                    }
                }
            }
            const int n = __reduce_add_sync(0xffffffffu, nsv);
            if (lane == 0 && n) atomicAdd(&scnt[q & 1], n);
            __syncwarp();
            if (lane == 0) mbar_arrive(&done[q & 1]);
        }
    }
    if (ok && B.st_mode) {
        // the last slice's cube-row words for the next push
#pragma unroll
        for (int i = 0; i < RY2; ++i) B.st_out[st_base + (long long)i * NC] = sst[i * NC];
    }
    if (!ok) atomicOr(status, ST_TIMEOUT);
    if (!EXACT) bad |= ((qa_and ^ MAGIC_BITS) | (qa_or ^ MAGIC_BITS)) & 0xFF800000u;
    if (bad & (EXACT ? 1u : 0xFF800000u)) atomicOr(status, EXACT ? ST_RANGE : ST_WIDE);
}

// ---- host side: launch configuration ----
size_t stream2_smem_bytes(int nx, int comps) { return (size_t)stream2_layout(nx, comps).total; }
int stream2_threads(int nx) { return stream2_consumers(nx) + 64; }

// rows up to 1024 floats: 192 threads, three CTAs per SM; up to 2048: up to
// 320; up to 4096: up to 576 (one CTA per SM).  Vector rows (two floats per
// vertex) up to 2048 vertices.
template <bool EXACT>
static void *stream2_kernel(int nx, int comps) {
    if (comps == 2) {
        if (nx <= 1024) return (void *)k_detect2_stream<EXACT, 192, 2, true>;
        return (void *)k_detect2_stream<EXACT, 320, 1, true>;
    }
    if (nx <= 1024) return (void *)k_detect2_stream<EXACT, 192, 3>;
    if (nx <= 2048) return (void *)k_detect2_stream<EXACT, 320, 1>;
    return (void *)k_detect2_stream<EXACT, 576, 1>;
}

long long stream2_state_words(const Field &F, const Blocking &B) {
    return (long long)B.nyb * RY2 * stream2_consumers(F.pitch);
}

int stream2_ctas_per_sm(int nx, int comps) {
    int n = 0;
    const size_t smem = stream2_smem_bytes(nx, comps);
    const void *k = stream2_kernel<false>(nx, comps);
    raise_smem_cap(k, smem, false);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, stream2_threads(nx), smem);
    return n > 0 ? n : 1;
}


cudaError_t launch_detect2(int variant, const Field &F, const Blocking &B, const Workspace &W, cudaStream_t s,
                           bool capturing) {
    const bool exact = variant == VAR_STREAM2_EXACT;
    const size_t smem = stream2_smem_bytes(F.pitch, F.comps);
    const void *k = exact ? stream2_kernel<true>(F.pitch, F.comps) : stream2_kernel<false>(F.pitch, F.comps);
    // the cap only ever grows: a graph may replay a wider field's launch
    // after a narrower one was configured
    const cudaError_t e = raise_smem_cap(k, smem, capturing);
    if (e != cudaSuccess) return e;
    const unsigned units = (unsigned)((long long)B.ntc * B.nyb);
    Field Fa = F;
    Blocking Ba = B;
    Workspace Wa = W;
    void *args[] = {&Fa, &Ba, &Wa};
    return cudaLaunchKernel(k, dim3(units), dim3(stream2_threads(F.pitch)), args, smem, s);
}

}  // namespace ftk
