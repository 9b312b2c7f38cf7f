// mbarrier and bulk-copy (TMA) helpers shared by the streaming detect
// kernels, as inline PTX for sm_103a.  Every wait is bounded.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ftk {

constexpr long long WAIT_CYCLES = 4000000000LL;   // bound of every mbarrier wait (~2 s)
constexpr uint32_t MAGIC_BITS = 0x4B400000u;      // bit pattern of 1.5 * 2^23
constexpr float MAGIC_F = 12582912.0f;            // 1.5 * 2^23

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on a phase; false if it did not complete within WAIT_CYCLES.
// Warps off the critical path (producer, compactor) back off with a sleep
// between polls (sleep_ns > 0), leaving the issue slots to the consumers.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned sleep_ns = 0) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > WAIT_CYCLES) return false;
        if (sleep_ns) __nanosleep(sleep_ns);
    }
    return true;
}
__device__ __forceinline__ void tma_row(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}


// CTA-wide named barrier over `threads` threads (a multiple of 32)
__device__ __forceinline__ void named_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Compactor of the streaming detect kernels (one warp): writes the set bits
// of words[0..nw) -- bit i stands for cube row i / nx, column i % nx of a
// segment -- as vertex ids (row0 + i / nx) * nx_ids + i % nx to out[pos..] in
// bit order (nx_ids = the grid's width, nx = the bitmap's row length), and
// clears the words.  A chunk of 32 * WPL words gives each lane
// WPL consecutive words, so a dense region spreads over the warp with one
// warp scan per chunk; chunks without a set bit are skipped.  inv_nx = 1 / nx
// (float); i < 2^24 keeps the row estimate within one of floor(i / nx), and
// the estimate is corrected.
template <int WPL>
__device__ __forceinline__ void compact_bits(uint32_t *words, int nw, int nx, int nx_ids, float inv_nx,
                                             long long row0, long long pos, long long *out, long long cap) {
    const int lane = threadIdx.x & 31;
    for (int k0 = 0; k0 < nw; k0 += 32 * WPL) {
        const int w0 = k0 + lane * WPL;
        uint32_t v[WPL];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < WPL; ++k) {
            v[k] = w0 + k < nw ? words[w0 + k] : 0u;
            cnt += __popc(v[k]);
        }
        if (!__ballot_sync(0xffffffffu, cnt != 0)) continue;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (cnt) {
            long long p = pos + incl - cnt;
            const int i0 = w0 * 32;
            int cr = __float2int_rz((float)i0 * inv_nx);
            if (cr * nx > i0) --cr;
            else if ((cr + 1) * nx <= i0) ++cr;
            int xw = i0 - cr * nx;      // column of the current word's bit 0
#pragma unroll
            for (int k = 0; k < WPL; ++k) {
                uint32_t bits = v[k];
                if (bits) words[w0 + k] = 0u;
                int x = xw, crr = cr, prev = 0;
                while (bits) {
                    const int bit = __ffs(bits) - 1;
                    bits &= bits - 1;
                    x += bit - prev;
                    prev = bit;
                    while (x >= nx) {
                        x -= nx;
                        ++crr;
                    }
                    if (p < cap) out[p] = (row0 + crr) * nx_ids + x;
                    ++p;
                }
                xw += 32;
                while (xw >= nx) {
                    xw -= nx;
                    ++cr;
                }
            }
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
}

}  // namespace ftk
