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
