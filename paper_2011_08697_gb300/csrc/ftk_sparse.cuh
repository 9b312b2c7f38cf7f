// Device helpers of the sparse stages shared by several translation units:
// samples, gradients and vertex coordinates read from global memory, and the
// exact evaluation of surviving 3D spacetime cubes (the faces each cube
// holds that the trajectory punctures, paper Sec. 4.3 with Eq. (1)).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ftk_device.cuh"
#include "ftk_kernels.cuh"

namespace ftk {

struct Pt { int c[4]; };   // x, y, z, t (z = 0 in 2D)

__device__ __forceinline__ int ext_of(const Field &F, int a) { return a == 0 ? F.nx : a == 1 ? F.ny : F.nz; }

// element offset of grid point p in the (row-padded) field, and the element
// stride of axis a (0 = x, 1 = y, 2 = z, 3 = t): samples around a point are
// addressed from its offset, not recomputed from coordinates
__device__ __forceinline__ long long vindex(const Field &F, const Pt &p) {
    return (((long long)p.c[3] * F.nz + p.c[2]) * F.ny + p.c[1]) * F.pitch + p.c[0];
}
__device__ __forceinline__ long long vstride(const Field &F, int a) {
    return a == 0 ? 1LL : a == 1 ? (long long)F.pitch : a == 2 ? (long long)F.ny * F.pitch
                                                            : (long long)F.nz * F.ny * F.pitch;
}
// quantised sample rint(f 2^S) at element i (0 outside the exact range,
// which the dense pass reports)
__device__ __forceinline__ int qat(const Field &F, long long i) {
    const float v = __ldg(F.f + i) * F.scale;
    return fabsf(v) <= RANGE_LIMIT ? __float2int_rn(v) : 0;
}

// gradient component a (spatial axis 0 = x, 1 = y, 2 = z) at point p of
// element offset ip: central difference f[p + e_a] - f[p - e_a], one-sided
// and doubled at either end of the axis, 2 (f[p + e_a] - f[p]) or
// 2 (f[p] - f[p - e_a]); equivalently, with the neighbours clamped into the
// grid, m_a (f[hi_a] - f[lo_a]) where m_a = 2 at an end, else 1.  a must be a
// compile-time constant after unrolling (p.c[a]).
__device__ __forceinline__ int grad_at(const Field &F, const Pt &p, long long ip, int a) {
    if (F.comps == 2) return qat(F, 2 * ip + a);   // a vector field: component a itself
    const int n = ext_of(F, a);
    const long long st = vstride(F, a);
    const long long lo = p.c[a] > 0 ? ip - st : ip;
    const long long hi = p.c[a] + 1 < n ? ip + st : ip;
    const int m = (p.c[a] == 0 || p.c[a] == n - 1) ? 2 : 1;
    return m * (qat(F, hi) - qat(F, lo));
}

// offset of vertex b + mask m from vertex b (axis N of m is time)
template <int N>
__device__ __forceinline__ long long mask_offset(const Field &F, int m) {
    long long o = (m & 1) + ((m >> 1) & 1) * (long long)F.pitch + ((m >> N) & 1) * vstride(F, 3);
    if (N == 3) o += ((m >> 2) & 1) * vstride(F, 2);
    return o;
}

// coordinates (x, y, z, t) of vertex id g
__device__ __forceinline__ Pt decode_vertex(const Field &F, long long g) {
    Pt p;
    if (F.small) {
        const unsigned u = (unsigned)g;
        const unsigned r1 = fdiv(u, F.dx);
        p.c[0] = (int)(u - r1 * (unsigned)F.nx);
        const unsigned r2 = fdiv(r1, F.dy);
        p.c[1] = (int)(r1 - r2 * (unsigned)F.ny);
        const unsigned r3 = fdiv(r2, F.dz);
        p.c[2] = (int)(r2 - r3 * (unsigned)F.nz);
        p.c[3] = (int)r3;
        return p;
    }
    p.c[0] = (int)(g % F.nx); g /= F.nx;
    p.c[1] = (int)(g % F.ny); g /= F.ny;
    p.c[2] = (int)(g % F.nz); g /= F.nz;
    p.c[3] = (int)g;
    return p;
}

template <int N>
__device__ __forceinline__ Pt add_mask(Pt p, int m) {
    p.c[0] += m & 1;
    p.c[1] += (m >> 1) & 1;
    if (N == 3) p.c[2] += (m >> 2) & 1;
    p.c[3] += (m >> N) & 1;
    return p;
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

// Exact SoS test of a 3D face whose three components each change sign over
// its vertices (the sign test that could exclude it has already failed):
// (-1)^k sign det(V without vertex k) equal for k = 0..3, int64 determinants
// when every entry fits
__device__ __forceinline__ bool face_punctured3_mixed(const int32_t (&V)[4][3]) {
    const bool fit = entries_fit20(V);
    int ref = 0;
#pragma unroll
    for (int k = 0; k <= 3; ++k) {
        int32_t M[3][3];
        int c = 0;
#pragma unroll
        for (int j = 0; j <= 3; ++j) {
            if (j == k) continue;
#pragma unroll
            for (int r = 0; r < 3; ++r) M[c][r] = V[j][r];
            ++c;
        }
        const int s = sos_det_sign3(M, fit);
        const int val = (k & 1) ? -s : s;
        if (k == 0) ref = val;
        else if (val != ref) return false;
    }
    return true;
}

// Per-lane constants of eval_pair3: the corner masks of face types lane and
// lane + 32 and the last mask of their chains.  fch[tt] = the chain of face
// type tt as m_1 | m_2 << 8 | m_3 << 16.
struct Pair3Lane {
    uint32_t M[2], last[2];
};
__device__ __forceinline__ Pair3Lane pair3_lane(const uint32_t *fch) {
    constexpr int T = MeshDims<3>::T;
    const int lane = threadIdx.x & 31;
    Pair3Lane L;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const int tt = f * 32 + lane;
        const uint32_t ch = tt < T ? fch[tt] : 0u;
        L.M[f] = tt < T ? (1u | 1u << (ch & 0xff) | 1u << ((ch >> 8) & 0xff) | 1u << (ch >> 16)) : 0u;
        L.last[f] = ch >> 16;
    }
    return L;
}

// Exact evaluation of surviving 3D cubes s0 and s0 + 1 of the survivor list
// (those below s_end), by one full warp: bit tt of W.surv_mask[s] = face type
// tt based at the cube's vertex is punctured.  Lanes 0-15 load the 16 corner
// gradients of the first cube, lanes 16-31 those of the second; three
// ballots give every corner's sign pattern.  A face whose corners agree in
// the sign of one component cannot be punctured (zero counts as positive:
// its perturbation is a positive infinitesimal); the faces of both cubes that
// pass this test are gathered and handed out one per lane for the exact SoS
// test.  Gs: this warp's shared [2][16][3] corner gradients.
__device__ __forceinline__ void eval_pair3(const Field &F, const Workspace &W, long long s0, long long s_end,
                                           int32_t (*Gs)[16][3], const uint32_t *fch, const Pair3Lane &L) {
    constexpr int N = 3, D = 4;
    constexpr uint32_t ALL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4, c = lane & 15;
    const long long s = s0 + half;
    const bool have = s < s_end;
    const long long g = have ? W.surv[s] : 0;
    const Pt b = decode_vertex(F, g);
    int inside = 0;   // bit a: axis a can step +1
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int slot = a == N ? 3 : a;
        const int ext = a == N ? F.nt : ext_of(F, a);
        if (b.c[slot] + 1 < ext) inside |= 1 << a;
    }
    if (!have) inside = 0;   // no face of a missing second cube is tested
    int32_t gc[N] = {};
    const bool corner = have && !(c & ~inside);
    if (corner) {
        const Pt p = add_mask<N>(b, c);
        const long long ip = vindex(F, b) + mask_offset<N>(F, c);
#pragma unroll
        for (int r = 0; r < N; ++r) gc[r] = grad_at(F, p, ip, r);
    }
#pragma unroll
    for (int r = 0; r < N; ++r) Gs[half][c][r] = gc[r];
    uint32_t neg[N];
#pragma unroll
    for (int r = 0; r < N; ++r) neg[r] = __ballot_sync(ALL, corner && gc[r] < 0);
    const int ins[2] = {__shfl_sync(ALL, inside, 0), __shfl_sync(ALL, inside, 16)};
    __syncwarp();
    // candidate lists: (cube q, face types 32 f + bit)
    uint32_t cand[4];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const uint32_t M = L.M[f];
            bool mixed = M != 0 && !(L.last[f] & ~ins[q]);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                const uint32_t nq = (neg[r] >> (16 * q)) & M;
                mixed &= nq != 0 && nq != M;
            }
            cand[2 * q + f] = __ballot_sync(ALL, mixed);
        }
    const int n0 = __popc(cand[0]), n1 = __popc(cand[1]), n2 = __popc(cand[2]);
    const int total = n0 + n1 + n2 + __popc(cand[3]);
    uint32_t mk[4] = {0u, 0u, 0u, 0u};   // punctured masks: cube 0 lo/hi, cube 1 lo/hi
    for (int j0 = 0; j0 < total; j0 += 32) {
        const int j = j0 + lane;
        int list = -1, bit = 0;
        if (j < total) {
            int n = j;
            list = n < n0 ? 0 : n < n0 + n1 ? 1 : n < n0 + n1 + n2 ? 2 : 3;
            n -= list == 0 ? 0 : list == 1 ? n0 : list == 2 ? n0 + n1 : n0 + n1 + n2;
            bit = nth_set_bit(list == 0 ? cand[0] : list == 1 ? cand[1] : list == 2 ? cand[2] : cand[3], n);
        }
        bool pun = false;
        if (list >= 0) {
            const int q = list >> 1;
            const uint32_t ch = fch[(list & 1) * 32 + bit];
            const int cr[4] = {0, (int)(ch & 0xff), (int)((ch >> 8) & 0xff), (int)(ch >> 16)};
            int32_t V[4][3];
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int r = 0; r < N; ++r) V[k][r] = Gs[q][cr[k]][r];
            pun = face_punctured3_mixed(V);
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) mk[l] |= __reduce_or_sync(ALL, pun && list == l ? 1u << bit : 0u);
    }
    if (have && c == 0)
        W.surv_mask[s] = half ? (unsigned long long)mk[2] | (unsigned long long)mk[3] << 32
                              : (unsigned long long)mk[0] | (unsigned long long)mk[1] << 32;
    __syncwarp();
}

}  // namespace ftk
