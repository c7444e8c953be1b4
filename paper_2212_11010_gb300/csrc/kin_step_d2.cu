// kin_step_d2.cu -- instantiations of the fused sweep + relaxation kernel for
// 2 space dimension(s), degrees 1..3, scalar advection and Euler, FP32/FP64.
#include "kin_aux.h"
#include "kin_device.cuh"
#include "kin_fixed.cuh"

namespace kin {

template <int P, int SYS>
static StepKernel pick(int prec)
{
    return prec == 1 ? (StepKernel)step_kernel<2, P, SYS, float>
                     : (StepKernel)step_kernel<2, P, SYS, double>;
}


// Fixed shapes compiled for 2D: (degree, system, precision, B0, B1, threads,
// min blocks per SM with one tile buffer, with two tile buffers).
#define KIN_FIXED_2D(X)                           \
    X(1, kEuler, float, 16, 8, 128, 6, 3)         \
    X(1, kEuler, float, 16, 16, 256, 3, 1)        \
    X(2, kEuler, float, 8, 8, 192, 5, 3)          \
    X(3, kEuler, float, 8, 4, 128, 6, 3)          \
    X(3, kEuler, float, 8, 8, 256, 3, 1)          \
    X(2, kEuler, double, 8, 8, 192, 3, 1)

FixedKernel fixed_kernel_d2(int degree, int system, int prec, const int B[3], int stages)
{
    FixedKernel k{nullptr, nullptr, 0, 0};
#define KIN_TRY(PP, SY, TT, X0, X1, NT, MB1, MB2)                                                  \
    if (degree == PP && system == SY && prec == (sizeof(TT) == 4 ? 1 : 0) && B[0] == X0 && B[1] == X1 && \
        B[2] == 1) {                                                                                \
        if (stages == 2) {                                                                          \
            k.fn = (StepKernel)step_kernel_fixed<2, PP, SY, TT, X0, X1, 1, NT, MB2, 2>;               \
            k.batch_fn = (const void*)step_kernel_fixed_batch<2, PP, SY, TT, X0, X1, 1, NT, MB2, 2>;  \
        } else {                                                                                    \
            k.fn = (StepKernel)step_kernel_fixed<2, PP, SY, TT, X0, X1, 1, NT, MB1, 1>;               \
            k.batch_fn = (const void*)step_kernel_fixed_batch<2, PP, SY, TT, X0, X1, 1, NT, MB1, 1>;  \
        }                                                                                           \
        k.threads = NT;                                                                             \
        k.smem = (stages == 2 ? 2 : 1) * Shape<2, PP, SY, TT, X0, X1, 1>::SMEM +                    \
                 Shape<2, PP, SY, TT, X0, X1, 1>::TIN_BYTES;                                          \
        return k;                                                                                   \
    }
    KIN_FIXED_2D(KIN_TRY)
#undef KIN_TRY
    return k;
}

// One-launch kernels for batches of 2D Euler FP32 problems of degrees 1..3:
// (threads, min blocks per SM, degree-1 block, degree-2 block, degree-3 block).
// The slots are the default blocks of each degree.  (Smaller blocks at five
// resident blocks of 192 threads, or four of 256, measured 35-45% slower on
// the 64-instance mix: the degree-3 sweeps need 80 registers.)
#define KIN_MIXED_2D(X) X(256, 3, 16, 16, 8, 8, 8, 8)

int mixed_kernels_2d(MixedKernel* out, int max)
{
    int n = 0;
#define KIN_MX(NT, MB, X0, X1, Y0, Y1, Z0, Z1)                                                  \
    if (n < max) {                                                                              \
        out[n].fn = (const void*)step_kernel_mixed2d<NT, MB, X0, X1, Y0, Y1, Z0, Z1>;             \
        out[n].threads = NT;                                                                    \
        out[n].min_blocks = MB;                                                                 \
        out[n].smem = Mixed2D<X0, X1, Y0, Y1, Z0, Z1>::SMEM;                                    \
        out[n].block[0][0] = X0;                                                                \
        out[n].block[0][1] = X1;                                                                \
        out[n].block[1][0] = Y0;                                                                \
        out[n].block[1][1] = Y1;                                                                \
        out[n].block[2][0] = Z0;                                                                \
        out[n].block[2][1] = Z1;                                                                \
        ++n;                                                                                    \
    }
    KIN_MIXED_2D(KIN_MX)
#undef KIN_MX
    return n;
}

StepKernel step_kernel_d2(int degree, int system, int prec)
{
    switch (degree * 4 + system) {        // (Maxwell is 3D only)
    case 4: return pick<1, kAdvection>(prec);
    case 5: return pick<1, kEuler>(prec);
    case 8: return pick<2, kAdvection>(prec);
    case 9: return pick<2, kEuler>(prec);
    case 12: return pick<3, kAdvection>(prec);
    case 13: return pick<3, kEuler>(prec);
    default: return nullptr;
    }
}

}  // namespace kin
