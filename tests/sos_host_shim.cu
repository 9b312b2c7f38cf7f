// Host build of the device determinant sign with Simulation of Simplicity,
// so that the CPU test-suite can compare it with the oracle's generic
// expansion (test support only; not part of the library).
#include <cstdint>

#include "../paper_2011_08697_gb300/csrc/ftk_device.cuh"

extern "C" int shim_sos_det_sign(int n, const int32_t *M) {
    if (n == 2) {
        const int32_t A[2][2] = {{M[0], M[1]}, {M[2], M[3]}};
        return ftk::sos_det_sign<2>(A);
    }
    int32_t A[3][3];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) A[c][r] = M[c * 3 + r];
    return ftk::sos_det_sign<3>(A);
}

// The FP32 Morse filters with the device's accumulation of S (one term per
// simplex vertex, weights scaled by a power of two).  w_k = (w_hi[k] << 64) |
// w_lo[k] as a two's complement 128-bit integer; hs: n+1 row-major n x n
// blocks of H_k + H_k^T.  Returns 1 and the index when the filter certifies
// it, else 0.
template <int N>
static int filter_n(const long long *w_hi, const unsigned long long *w_lo, const long long *hs, int *morse) {
    __int128 w[N + 1], wmax = 0;
    for (int k = 0; k <= N; ++k) {
        w[k] = (__int128)(((unsigned __int128)(unsigned long long)w_hi[k] << 64) | w_lo[k]);
        const __int128 a = w[k] < 0 ? -w[k] : w[k];
        if (a > wmax) wmax = a;
    }
    const int wbits = ftk::i128_bits(wmax);
    float Sd[N][N] = {}, Ad[N][N] = {};
    for (int k = 0; k <= N; ++k) {
        long long HS[N][N];
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) HS[a][b] = hs[(k * N + a) * N + b];
        ftk::s_fp32_step<N>(ldexpf(ftk::i128_to_float(w[k]), 1 - wbits), HS, Sd, Ad);
    }
    ftk::s_fp32_symmetrise<N>(Sd, Ad);
    int m = 0;
    bool ok;
    if constexpr (N == 2) ok = ftk::morse_filter2(Sd, Ad, m);
    else ok = ftk::morse_filter3(Sd, Ad, m);
    *morse = m;
    return ok ? 1 : 0;
}

extern "C" int shim_morse_filter(int n, const long long *w_hi, const unsigned long long *w_lo, const long long *hs,
                                 int *morse) {
    return n == 2 ? filter_n<2>(w_hi, w_lo, hs, morse) : filter_n<3>(w_hi, w_lo, hs, morse);
}

// The CUDA path's mesh tables: face chains in type order (T x n masks) and,
// per cell type, the bit set of its sides through the base vertex, the type
// of the side opposite it and the axis of the cell's first step.
extern "C" int shim_face_chains(int n, int *out) {
    if (n == 2) {
        const ftk::MeshTables<2> t;
        for (int i = 0; i < ftk::MeshDims<2>::T; ++i)
            for (int k = 0; k < 2; ++k) out[i * 2 + k] = t.face[i][k];
        return ftk::MeshDims<2>::T;
    }
    const ftk::MeshTables<3> t;
    for (int i = 0; i < ftk::MeshDims<3>::T; ++i)
        for (int k = 0; k < 3; ++k) out[i * 3 + k] = t.face[i][k];
    return ftk::MeshDims<3>::T;
}

extern "C" int shim_cell_table(int n, unsigned long long *own, int *far, int *axis) {
    if (n == 2) {
        const ftk::CellTables<2> c;
        for (int i = 0; i < ftk::MeshDims<2>::C; ++i) { own[i] = c.own[i]; far[i] = c.far[i]; axis[i] = c.axis[i]; }
        return ftk::MeshDims<2>::C;
    }
    const ftk::CellTables<3> c;
    for (int i = 0; i < ftk::MeshDims<3>::C; ++i) { own[i] = c.own[i]; far[i] = c.far[i]; axis[i] = c.axis[i]; }
    return ftk::MeshDims<3>::C;
}

// The segment of a vertex (the runs of face ids the compaction and the
// sparse stages address by segment), with and without x windows: from the
// vertex id (FastDiv path when small, else 64-bit division) and from its
// coordinates.  out[0] = segment_of(g), out[1] = segment_of_coords(...),
// out[2] = segment_count.
#include "../paper_2011_08697_gb300/csrc/ftk_kernels.cuh"

extern "C" void shim_segment(int nx, int ny, int nz, int nt, int ry, int nxb, int wx, int small, long long g,
                             long long *out) {
    ftk::Field F{};
    F.nx = nx; F.ny = ny; F.nz = nz; F.nt = nt; F.pitch = nx;
    ftk::field_divisors(F);
    F.small = small && F.small;
    ftk::Blocking B{};
    B.ry = ry;
    B.nyb = (ny + ry - 1) / ry;
    B.nxb = nxb;
    B.wx = wx;
    long long r = g;
    const int x = (int)(r % nx); r /= nx;
    const int y = (int)(r % ny); r /= ny;
    const int z = (int)(r % nz); r /= nz;
    const int t = (int)r;
    out[0] = ftk::segment_of(g, F, B);
    out[1] = ftk::segment_of_coords(x, y, z, t, F, B);
    out[2] = ftk::segment_count(F, B);
}
