// Device building blocks of the GB300 critical-point tracker.
//
//  * MeshTables<N>: the implicit simplicial spacetime mesh of a regular grid
//    (paper Sec. 3.3).  Each unit (N+1)-cube is split into (N+1)! simplices
//    (monotone chains of axis flips, the "recursive extrusion" of Sec. 3.3 /
//    Table 1); a k-simplex is a base vertex plus a strictly nested chain of
//    k nonempty axis bitmasks.  Face (N-simplex) types are ranked in
//    lexicographic chain order; the tables are generated at compile time.
//  * Exact puncture predicate (Sec. 4.3, Eq. 1): 0 lies in the interior of
//    the simplex spanned by the N+1 gradient vectors iff the signed
//    determinants (-1)^k det(V without column k) all agree.  Determinants
//    are exact (int64 in 2D, int128 in 3D).  Zero determinants are decided
//    by Simulation of Simplicity: entry (row r, column c) of a determinant
//    whose columns are sorted by global vertex id is perturbed by
//    eps^(2^(c*N + r)); the sign is that of the first nonzero coefficient
//    in increasing exponent order, written out term by term for N = 2, 3.
//  * BigInt<W>: fixed-width two's-complement integers for the exact Morse
//    classification (products up to ~2^390 in 3D).
#pragma once
#include <cmath>
#include <cstdint>

namespace ftk {

// ----------------------------------------------------------------------------
// Mesh tables
// ----------------------------------------------------------------------------
template <int N>
struct MeshDims {
    static constexpr int D = N + 1;                 // spacetime dimension
    static constexpr int FULL = (1 << D) - 1;
    static constexpr int TBIT = 1 << N;             // time axis bit
    static constexpr int T = (N == 2) ? 12 : 60;    // face (N-simplex) types per vertex
    static constexpr int C = (N == 2) ? 6 : 24;     // cell ((N+1)-simplex) types
};

template <int N>
struct MeshTables {
    using M = MeshDims<N>;
    uint8_t face[M::T][N];        // face chains m_1..m_N
    uint8_t lookup[1 << (4 * N)]; // chain key (4 bits per mask) -> type, 255 if none

    __host__ __device__ constexpr MeshTables() : face{}, lookup{} {
        for (int i = 0; i < (1 << (4 * N)); ++i) lookup[i] = 255;
        // odometer over (m_1, .., m_N) in [1, FULL]^N in lexicographic order,
        // keeping strictly nested chains; the visiting order is the rank order
        int idx[N] = {};
        for (int i = 0; i < N; ++i) idx[i] = 1;
        int cnt = 0;
        while (true) {
            bool ok = true;
            int prev = 0;
            for (int i = 0; i < N; ++i) {
                const int m = idx[i];
                if ((m & prev) != prev || m == prev) { ok = false; break; }
                prev = m;
            }
            if (ok) {
                int key = 0;
                for (int i = 0; i < N; ++i) {
                    face[cnt][i] = (uint8_t)idx[i];
                    key |= idx[i] << (4 * i);
                }
                lookup[key] = (uint8_t)cnt;
                ++cnt;
            }
            int p = N - 1;
            while (p >= 0 && idx[p] == M::FULL) { idx[p] = 1; --p; }
            if (p < 0) break;
            ++idx[p];
        }
    }
};

// Cells ((N+1)-simplices) of one unit cube, one per order in which the axes
// are stepped: chain m_0 < m_1 < .. < m_N = FULL from the base vertex b.  Of
// a cell's N+2 sides, the N+1 through b are faces based at b (drop vertex
// b + m_k: chain without m_k); the side opposite b is based at b + m_0 with
// chain (m_1 ^ m_0, .., m_N ^ m_0), i.e. a face of the next cube along the
// first step's axis.
template <int N>
struct CellTables {
    using M = MeshDims<N>;
    // cells are ordered by the axis of their first step: cells
    // [a C / (N+1), (a+1) C / (N+1)) step first along axis a
    unsigned long long own[M::C];   // bit set of the types of the sides through b
    unsigned long long own_axis[M::D];  // union of own[] over the cells of one first axis
    uint8_t side[M::C][N + 1];      // those types, side k dropping vertex b + m_k
    uint8_t far[M::C];              // type of the side opposite b
    uint8_t axis[M::C];             // axis of the first step

    __host__ __device__ constexpr CellTables() : own{}, own_axis{}, side{}, far{}, axis{} {
        const MeshTables<N> mt;
        constexpr int D = M::D;
        int tuples = 1;
        for (int i = 0; i < D; ++i) tuples *= D;
        int cnt = 0;
        for (int code = 0; code < tuples; ++code) {
            int p[D] = {};
            int c = code, used = 0;
            bool ok = true;
            for (int j = D - 1; j >= 0; --j) {   // p[0] is the slowest digit
                p[j] = c % D;
                c /= D;
                if ((used >> p[j]) & 1) ok = false;
                used |= 1 << p[j];
            }
            if (!ok) continue;
            int m[D] = {};
            int acc = 0;
            for (int j = 0; j < D; ++j) {
                acc |= 1 << p[j];
                m[j] = acc;
            }
            unsigned long long bits = 0;
            for (int k = 0; k < D; ++k) {
                int key = 0, w = 0;
                for (int j = 0; j < D; ++j)
                    if (j != k) key |= m[j] << (4 * w++);
                side[cnt][k] = mt.lookup[key];
                bits |= 1ull << mt.lookup[key];
            }
            own[cnt] = bits;
            own_axis[p[0]] |= bits;
            int key = 0;
            for (int j = 1; j < D; ++j) key |= (m[j] ^ m[0]) << (4 * (j - 1));
            far[cnt] = mt.lookup[key];
            axis[cnt] = (uint8_t)p[0];
            ++cnt;
        }
    }
};

template <int N>
__host__ __device__ constexpr int chain_key(const int (&m)[N]) {
    int key = 0;
    for (int i = 0; i < N; ++i) key |= m[i] << (4 * i);
    return key;
}

// ----------------------------------------------------------------------------
// Floating-point filters of the Morse classification (host and device, so
// that the CPU tests can check them against exact arithmetic)
// ----------------------------------------------------------------------------
// fused multiply-add rounded once to nearest, on either side
__host__ __device__ inline float fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}

// bit length of |w| (1 for w = 0): the scale 2^(1 - bits) maps the largest
// weight into [1, 2)
__host__ __device__ inline int i128_bits(__int128 w) {
    const unsigned __int128 u = w < 0 ? (unsigned __int128)(-w) : (unsigned __int128)w;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
#ifdef __CUDA_ARCH__
    return hi ? 128 - __clzll((long long)hi) : (lo ? 64 - __clzll((long long)lo) : 1);
#else
    return hi ? 128 - __builtin_clzll(hi) : (lo ? 64 - __builtin_clzll(lo) : 1);
#endif
}

__host__ __device__ inline float i128_to_float(__int128 v) {
    const bool neg = v < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    const float r = fma_rn((float)hi, 18446744073709551616.0f, (float)lo);
    return neg ? -r : r;
}

// Morse index of the symmetric 2x2 S from an FP32 evaluation, when its signs
// are certain (same error model as the 3x3 filter below: Sd from weights
// scaled by a power of two, every entry within e = 16u Ad + 2^-90 of the
// scaled exact value; the perturbation bound of a product of two entries is
// M_i M_j - |Sd_i| |Sd_j| with M = |Sd| + e, plus its own rounding).
// det S < 0: saddle (1); det S > 0: maximum (2) if tr S < 0, else minimum (0).
__host__ __device__ inline bool morse_filter2(const float (&Sd)[2][2], const float (&Ad)[2][2], int &morse) {
    const float u = 5.9604644775390625e-8f;   // 2^-24
    const float floor_abs = 8.0779356e-28f;   // 2^-90
    float e[2][2], a[2][2], M[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            e[i][j] = 16.0f * u * Ad[i][j] + floor_abs;
            a[i][j] = fabsf(Sd[i][j]);
            M[i][j] = a[i][j] + e[i][j];
        }
    const float det = Sd[0][0] * Sd[1][1] - Sd[0][1] * Sd[0][1];
    const float err_det = (M[0][0] * M[1][1] - a[0][0] * a[1][1]) + (M[0][1] * M[0][1] - a[0][1] * a[0][1]) +
                          4.0f * u * (M[0][0] * M[1][1] + M[0][1] * M[0][1]);
    // every comparison is false for a non-finite value: then the exact path
    if (!(fabsf(det) > 2.0f * err_det)) return false;
    if (det < 0.0f) {
        morse = 1;
        return true;
    }
    const float tr = Sd[0][0] + Sd[1][1];
    const float err_tr = (e[0][0] + e[1][1]) + 2.0f * u * (M[0][0] + M[1][1]);
    if (!(fabsf(tr) > 2.0f * err_tr)) return false;
    morse = tr < 0.0f ? 2 : 0;
    return true;
}

// Morse index of the symmetric 3x3 S from an FP32 evaluation, when its
// signs are certain (the index is unchanged by a positive scale of S, so the
// weights come in scaled by a power of two into [1, 2) for the largest).
// Sd = S evaluated in FP32 from the scaled weights and the exact int64
// Hessian sums: conversion, product and a 4-term sum stay within
// 9u sum_k |w_k h_k| of the exact scaled entry, u = 2^-24; denormal
// rounding adds at most 2^-100 absolutely.  Ad = sum_k |w_k h_k| in FP32.
// With e = 16u Ad + 2^-90 bounding each entry's error and M = |Sd| + e
// bounding each exact entry, the errors of tr, m2 and det are bounded by the
// change of each monomial under the entry perturbations (prod M - prod |Sd|)
// plus the rounding of their evaluation.  Returns false (the caller decides
// exactly) unless every invariant exceeds twice its bound.
__host__ __device__ inline bool morse_filter3(const float (&Sd)[3][3], const float (&Ad)[3][3], int &morse) {
    const float u = 5.9604644775390625e-8f;   // 2^-24
    const float floor_abs = 8.0779356e-28f;   // 2^-90
    float e[3][3], M[3][3], a[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            e[i][j] = 16.0f * u * Ad[i][j] + floor_abs;
            a[i][j] = fabsf(Sd[i][j]);
            M[i][j] = a[i][j] + e[i][j];
        }
    const float tr = Sd[0][0] + Sd[1][1] + Sd[2][2];
    const float err_tr = (e[0][0] + e[1][1] + e[2][2]) + 4.0f * u * (M[0][0] + M[1][1] + M[2][2]);
    float m2 = 0.0f, err_m2 = 0.0f, mag_m2 = 0.0f;
    const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int i = P[q][0], j = P[q][1];
        m2 += Sd[i][i] * Sd[j][j] - Sd[i][j] * Sd[i][j];
        err_m2 += (M[i][i] * M[j][j] - a[i][i] * a[j][j]) + (M[i][j] * M[i][j] - a[i][j] * a[i][j]);
        mag_m2 += M[i][i] * M[j][j] + M[i][j] * M[i][j];
    }
    err_m2 += 8.0f * u * mag_m2;
    const float c0 = Sd[1][1] * Sd[2][2] - Sd[1][2] * Sd[2][1];
    const float c1 = Sd[1][0] * Sd[2][2] - Sd[1][2] * Sd[2][0];
    const float c2 = Sd[1][0] * Sd[2][1] - Sd[1][1] * Sd[2][0];
    const float det = Sd[0][0] * c0 - Sd[0][1] * c1 + Sd[0][2] * c2;
    // the six monomials of det: perturbation bound and magnitude
    const int pm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    float err_det = 0.0f, mag_det = 0.0f;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float Mp = M[0][pm[q][0]] * M[1][pm[q][1]] * M[2][pm[q][2]];
        const float ap = a[0][pm[q][0]] * a[1][pm[q][1]] * a[2][pm[q][2]];
        err_det += Mp - ap;
        mag_det += Mp;
    }
    err_det += 12.0f * u * mag_det;
    // every comparison is false for a non-finite value: then the exact path
    if (!(fabsf(tr) > 2.0f * err_tr && fabsf(m2) > 2.0f * err_m2 && fabsf(det) > 2.0f * err_det)) return false;
    const int s[3] = {tr > 0.0f ? 1 : -1, m2 > 0.0f ? 1 : -1, det > 0.0f ? 1 : -1};
    int prev = 1, changes = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (s[i] != prev) ++changes;
        prev = s[i];
    }
    morse = changes;
    return true;
}

// one vertex's term of S in FP32: Sd += wd HS, Ad += |wd| |HS| (upper
// triangle), wd = the vertex's weight scaled by a power of two
template <int N>
__host__ __device__ inline void s_fp32_step(float wd, const long long (&HS)[N][N], float (&Sd)[N][N],
                                            float (&Ad)[N][N]) {
    const float aw = fabsf(wd);
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = a; b < N; ++b) {
            const float hd = (float)HS[a][b];
            Sd[a][b] = fma_rn(wd, hd, Sd[a][b]);
            Ad[a][b] = fma_rn(aw, fabsf(hd), Ad[a][b]);
        }
}
template <int N>
__host__ __device__ inline void s_fp32_symmetrise(float (&Sd)[N][N], float (&Ad)[N][N]) {
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < a; ++b) {
            Sd[a][b] = Sd[b][a];
            Ad[a][b] = Ad[b][a];
        }
}

// ----------------------------------------------------------------------------
// Exact determinants and the SoS sign
// ----------------------------------------------------------------------------
__device__ __forceinline__ int sgn128(__int128 v) { return (v > 0) - (v < 0); }

// M[c][r]: column c = vertex (sorted by id), row r = vector component
__host__ __device__ __forceinline__ __int128 det_exact(const int32_t (&M)[2][2]) {
    return (__int128)((int64_t)M[0][0] * M[1][1] - (int64_t)M[0][1] * M[1][0]);
}
__host__ __device__ __forceinline__ __int128 det_exact(const int32_t (&M)[3][3]) {
    // expansion along the first component row; 2x2 minors fit in int64
    const int64_t m0 = (int64_t)M[1][1] * M[2][2] - (int64_t)M[1][2] * M[2][1];
    const int64_t m1 = (int64_t)M[0][1] * M[2][2] - (int64_t)M[0][2] * M[2][1];
    const int64_t m2 = (int64_t)M[0][1] * M[1][2] - (int64_t)M[0][2] * M[1][1];
    return (__int128)M[0][0] * m0 - (__int128)M[1][0] * m1 + (__int128)M[2][0] * m2;
}

// Sign of det(M + E(eps)) when det(M) = 0 (Simulation of Simplicity, Sec. 4.1;
// Edelsbrunner-Muecke form): entry M[c][r] is perturbed by eps^(2^(c N + r)),
// so every set S of perturbed entries has its own exponent sum_{S} 2^(c N + r)
// and the sign is that of the first nonzero coefficient in increasing
// exponent order.  A set contributes only if it is a partial permutation
// (distinct columns and rows); its coefficient is the signed sum over the
// permutations through S of the unperturbed entries.  In that order the
// terms are: single entries (coefficient = cofactor), pairs (coefficient =
// +-the remaining entry) and, at the latest with a full permutation,
// a constant +-1.  Written out term by term for N = 2 and N = 3:
__host__ __device__ __forceinline__ int sgn_nz(long long v) { return v > 0 ? 1 : -1; }

__host__ __device__ __forceinline__ int sos_zero_sign(const int32_t (&M)[2][2]) {
    // masks 1 {(0,0)}, 2 {(0,1)}, 4 {(1,0)}, 6 {(0,1),(1,0)}
    if (M[1][1]) return sgn_nz(M[1][1]);
    if (M[1][0]) return -sgn_nz(M[1][0]);
    if (M[0][1]) return -sgn_nz(M[0][1]);
    return -1;
}

__host__ __device__ __forceinline__ int sos_zero_sign(const int32_t (&M)[3][3]) {
    typedef long long ll;
    ll v;
    // masks 1, 2, 4, 8: cofactors of (c,r) = (0,0), (0,1), (0,2), (1,0)
    if ((v = (ll)M[1][1] * M[2][2] - (ll)M[1][2] * M[2][1])) return sgn_nz(v);
    if ((v = (ll)M[1][2] * M[2][0] - (ll)M[1][0] * M[2][2])) return sgn_nz(v);
    if ((v = (ll)M[1][0] * M[2][1] - (ll)M[1][1] * M[2][0])) return sgn_nz(v);
    if ((v = (ll)M[0][2] * M[2][1] - (ll)M[0][1] * M[2][2])) return sgn_nz(v);
    // mask 10 {(0,1),(1,0)}: -M[2][2]; mask 12 {(0,2),(1,0)}: +M[2][1]
    if (M[2][2]) return -sgn_nz(M[2][2]);
    if (M[2][1]) return sgn_nz(M[2][1]);
    // mask 16: cofactor of (1,1)
    if ((v = (ll)M[0][0] * M[2][2] - (ll)M[0][2] * M[2][0])) return sgn_nz(v);
    // mask 17 {(0,0),(1,1)}: +M[2][2] (zero here); mask 20 {(0,2),(1,1)}: -M[2][0]
    if (M[2][0]) return -sgn_nz(M[2][0]);
    // mask 32: cofactor of (1,2); masks 33 (-M[2][1]) and 34 (+M[2][0]) are zero here
    if ((v = (ll)M[0][1] * M[2][0] - (ll)M[0][0] * M[2][1])) return sgn_nz(v);
    // mask 64: cofactor of (2,0)
    if ((v = (ll)M[0][1] * M[1][2] - (ll)M[0][2] * M[1][1])) return sgn_nz(v);
    // mask 66 {(0,1),(2,0)}: +M[1][2]; mask 68 {(0,2),(2,0)}: -M[1][1];
    // mask 80 {(1,1),(2,0)}: -M[0][2]; mask 84 {(0,2),(1,1),(2,0)}: -1
    if (M[1][2]) return sgn_nz(M[1][2]);
    if (M[1][1]) return -sgn_nz(M[1][1]);
    if (M[0][2]) return -sgn_nz(M[0][2]);
    return -1;
}

// true iff every entry lies in [-2^20, 2^20): then a 3x3 determinant is
// exact in int64 (2x2 minors below 2^41, each entry-times-minor product at
// most 2^61, their sum below 3 * 2^61 < 2^63)
template <int R, int C>
__host__ __device__ __forceinline__ bool entries_fit20(const int32_t (&V)[R][C]) {
    unsigned acc = 0;
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < C; ++j) acc |= (unsigned)(V[i][j] + (1 << 20));
    return acc < (1u << 21);
}

// sign of det M for entries in [-2^20, 2^20), the expansion of det_exact in int64
__host__ __device__ __forceinline__ int det3_sign64(const int32_t (&M)[3][3]) {
    const int64_t m0 = (int64_t)M[1][1] * M[2][2] - (int64_t)M[1][2] * M[2][1];
    const int64_t m1 = (int64_t)M[0][1] * M[2][2] - (int64_t)M[0][2] * M[2][1];
    const int64_t m2 = (int64_t)M[0][1] * M[1][2] - (int64_t)M[0][2] * M[1][1];
    const int64_t d = (int64_t)M[0][0] * m0 - (int64_t)M[1][0] * m1 + (int64_t)M[2][0] * m2;
    return (d > 0) - (d < 0);
}

// SoS sign of a 3x3 determinant whose entries are known to fit (or not) the
// int64 range of det3_sign64
__host__ __device__ __forceinline__ int sos_det_sign3(const int32_t (&M)[3][3], bool fit20) {
    if (fit20) {
        const int s = det3_sign64(M);
        return s != 0 ? s : sos_zero_sign(M);
    }
    const __int128 d = det_exact(M);
    if (d != 0) return d > 0 ? 1 : -1;
    return sos_zero_sign(M);
}

template <int N>
__host__ __device__ __forceinline__ int sos_det_sign(const int32_t (&M)[N][N]) {
    if constexpr (N == 3) return sos_det_sign3(M, entries_fit20(M));
    const __int128 d = det_exact(M);
    if (d != 0) return d > 0 ? 1 : -1;
    return sos_zero_sign(M);
}

// ----------------------------------------------------------------------------
// Fixed-width two's-complement big integers (little-endian 32-bit limbs)
// ----------------------------------------------------------------------------
template <int W>
struct BigInt {
    uint32_t w[W];
};

template <int W>
__device__ __forceinline__ BigInt<W> big_from(__int128 v) {
    BigInt<W> r;
    const uint32_t fill = v < 0 ? 0xffffffffu : 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        r.w[i] = i < 4 ? (uint32_t)((unsigned __int128)v >> (32 * i)) : fill;
    }
    return r;
}

template <int W>
__device__ __forceinline__ BigInt<W> big_add(const BigInt<W> &a, const BigInt<W> &b) {
    BigInt<W> r;
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t s = (uint64_t)a.w[i] + b.w[i] + c;
        r.w[i] = (uint32_t)s;
        c = s >> 32;
    }
    return r;
}

template <int W>
__device__ __forceinline__ BigInt<W> big_sub(const BigInt<W> &a, const BigInt<W> &b) {
    BigInt<W> r;
    uint64_t borrow = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t s = (uint64_t)a.w[i] - b.w[i] - borrow;
        r.w[i] = (uint32_t)s;
        borrow = (s >> 32) & 1;
    }
    return r;
}

// product modulo 2^(32W); exact whenever the signed product fits in W limbs
template <int W>
__device__ __forceinline__ BigInt<W> big_mul(const BigInt<W> &a, const BigInt<W> &b) {
    BigInt<W> r;
#pragma unroll
    for (int i = 0; i < W; ++i) r.w[i] = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        uint64_t c = 0;
#pragma unroll
        for (int j = 0; i + j < W; ++j) {
            const uint64_t t = (uint64_t)a.w[i] * b.w[j] + r.w[i + j] + c;
            r.w[i + j] = (uint32_t)t;
            c = t >> 32;
        }
    }
    return r;
}

template <int W>
__device__ __forceinline__ int big_sign(const BigInt<W> &a) {
    if (a.w[W - 1] >> 31) return -1;
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) any |= a.w[i];
    return any ? 1 : 0;
}

}  // namespace ftk
