// kin_step_d1.cu -- instantiations of the fused sweep + relaxation kernel for
// 1 space dimension(s), degrees 1..3, scalar advection and Euler, FP32/FP64.
#include "kin_aux.h"
#include "kin_device.cuh"

namespace kin {

template <int P, int SYS>
static StepKernel pick(int prec)
{
    return prec == 1 ? (StepKernel)step_kernel<1, P, SYS, float>
                     : (StepKernel)step_kernel<1, P, SYS, double>;
}

StepKernel step_kernel_d1(int degree, int system, int prec)
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
