// kin_step_d3.cu -- instantiations of the fused sweep + relaxation kernel for
// 3 space dimension(s), degrees 1..3, scalar advection, Euler and Maxwell, FP32/FP64.
#include "kin_aux.h"
#include "kin_device.cuh"
#include "kin_fixed.cuh"

namespace kin {

template <int P, int SYS>
static StepKernel pick(int prec)
{
    return prec == 1 ? (StepKernel)step_kernel<3, P, SYS, float>
                     : (StepKernel)step_kernel<3, P, SYS, double>;
}


// Fixed shapes compiled for 3D: (degree, system, precision, B0, B1, B2,
// threads, min blocks per SM with one tile buffer, with two tile buffers).
#define KIN_FIXED_3D(X)                             \
    X(1, kEuler, float, 8, 2, 2, 128, 6, 3)         \
    X(1, kEuler, float, 4, 4, 2, 128, 6, 3)         \
    X(1, kEuler, float, 8, 4, 2, 256, 3, 1)         \
    X(1, kEuler, float, 4, 4, 4, 320, 3, 1)         \
    X(1, kMaxwell, float, 4, 4, 2, 128, 4, 2)       \
    X(1, kMaxwell, float, 8, 2, 2, 128, 4, 2)       \
    X(1, kMaxwell, float, 4, 2, 2, 64, 8, 4)        \
    X(1, kMaxwell, float, 8, 4, 2, 256, 2, 1)       \
    X(1, kMaxwell, float, 4, 4, 4, 256, 2, 1)

FixedKernel fixed_kernel_d3(int degree, int system, int prec, const int B[3], int stages)
{
    FixedKernel k{nullptr, nullptr, 0, 0};
#define KIN_TRY(PP, SY, TT, X0, X1, X2, NT, MB1, MB2)                                              \
    if (degree == PP && system == SY && prec == (sizeof(TT) == 4 ? 1 : 0) && B[0] == X0 && B[1] == X1 && \
        B[2] == X2) {                                                                               \
        if (stages == 2) {                                                                          \
            k.fn = (StepKernel)step_kernel_fixed<3, PP, SY, TT, X0, X1, X2, NT, MB2, 2>;              \
            k.batch_fn = (const void*)step_kernel_fixed_batch<3, PP, SY, TT, X0, X1, X2, NT, MB2, 2>; \
        } else {                                                                                    \
            k.fn = (StepKernel)step_kernel_fixed<3, PP, SY, TT, X0, X1, X2, NT, MB1, 1>;              \
            k.batch_fn = (const void*)step_kernel_fixed_batch<3, PP, SY, TT, X0, X1, X2, NT, MB1, 1>; \
        }                                                                                           \
        k.threads = NT;                                                                             \
        k.smem = (stages == 2 ? 2 : 1) * Shape<3, PP, SY, TT, X0, X1, X2>::SMEM +                   \
                 Shape<3, PP, SY, TT, X0, X1, X2>::TIN_BYTES;                                         \
        return k;                                                                                   \
    }
    KIN_FIXED_3D(KIN_TRY)
#undef KIN_TRY
    return k;
}

// One tile buffer: the two-buffer schedule halves the resident blocks, and
// the loads of one block are already hidden behind the other blocks' work
// (measured slower for every compiled shape).
int fixed_default_stages(int, int, int, int, const int*) { return 1; }

int fixed_shapes(int dim, int degree, int system, int prec, int out[4][3])
{
    int n = 0;
    auto add = [&](int a, int b, int c) {
        if (n < 4) {
            out[n][0] = a;
            out[n][1] = b;
            out[n][2] = c;
            ++n;
        }
    };
    if (system == kMaxwell) {
        if (dim == 3 && prec == 1 && degree == 1) {
            add(4, 4, 4);
            add(4, 4, 2);
            add(8, 2, 2);
            add(4, 2, 2);
        }
        return n;
    }
    if (system != kEuler) return 0;
    if (dim == 2 && prec == 1) {
        if (degree == 1) {
            add(16, 16, 1);
            add(16, 8, 1);
        }
        if (degree == 2) add(8, 8, 1);
        if (degree == 3) {
            add(8, 8, 1);
            add(8, 4, 1);
        }
    }
    if (dim == 2 && prec == 0 && degree == 2) add(8, 8, 1);
    if (dim == 3 && prec == 1 && degree == 1) {
        add(4, 4, 4);
        add(8, 4, 2);
        add(4, 4, 2);
        add(8, 2, 2);
    }
    return n;
}

StepKernel step_kernel_d3(int degree, int system, int prec)
{
    switch (degree * 4 + system) {
    case 4: return pick<1, kAdvection>(prec);
    case 5: return pick<1, kEuler>(prec);
    case 6: return pick<1, kMaxwell>(prec);
    case 8: return pick<2, kAdvection>(prec);
    case 9: return pick<2, kEuler>(prec);
    case 10: return pick<2, kMaxwell>(prec);
    case 12: return pick<3, kAdvection>(prec);
    case 13: return pick<3, kEuler>(prec);
    case 14: return pick<3, kMaxwell>(prec);
    default: return nullptr;
    }
}

}  // namespace kin
