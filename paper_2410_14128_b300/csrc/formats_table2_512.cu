// formats_table2_512.cu -- compile-time-composed kernels for the 512^3
// formats of Table 2 that the other files do not already hold (labels 21-40;
// 24 and 28-30 live in formats_small.cu).
#include "trace.cuh"

namespace vx {
namespace {
#define VX_FMT(id, text, ...)                                                     \
    const KernelSet ks_##id = make_kernel_set<Format<__VA_ARGS__>>(text);        \
    KernelSetRegistrar reg_##id(&ks_##id);

VX_FMT(t21, "D(3,3,3,6) D(3,3,3,6) G(3)", Df<3, 3, 3, 6>, Df<3, 3, 3, 6>, Dag<3>)
VX_FMT(t22, "D(3,3,3,6) R(3,3,3) G(3)", Df<3, 3, 3, 6>, Raw<3, 3, 3>, Dag<3>)
VX_FMT(t23, "R(3,3,3) R(3,3,3) G(3)", Raw<3, 3, 3>, Raw<3, 3, 3>, Dag<3>)
VX_FMT(t25, "R(4,4,4) R(1,1,1) R(4,4,4)", Raw<4, 4, 4>, Raw<1, 1, 1>, Raw<4, 4, 4>)
VX_FMT(t26, "D(4,4,4,6) S(5)", Df<4, 4, 4, 6>, Svo<5>)
VX_FMT(t27, "D(4,4,4,6) G(5)", Df<4, 4, 4, 6>, Dag<5>)
VX_FMT(t31, "R(7,7,7) G(2)", Raw<7, 7, 7>, Dag<2>)
VX_FMT(t32, "S(5) R(4,4,4)", Svo<5>, Raw<4, 4, 4>)
VX_FMT(t33, "G(5) R(4,4,4)", Dag<5>, Raw<4, 4, 4>)
VX_FMT(t34, "D(5,5,5,6) D(4,4,4,6)", Df<5, 5, 5, 6>, Df<4, 4, 4, 6>)
VX_FMT(t35, "D(5,5,5,6) R(4,4,4)", Df<5, 5, 5, 6>, Raw<4, 4, 4>)
VX_FMT(t36, "R(5,5,5) R(4,4,4)", Raw<5, 5, 5>, Raw<4, 4, 4>)
VX_FMT(t37, "R(9,9,9)", Raw<9, 9, 9>)
VX_FMT(t38, "D(9,9,9,6)", Df<9, 9, 9, 6>)
VX_FMT(t39, "S(9)", Svo<9>)
VX_FMT(t40, "G(9)", Dag<9>)
#undef VX_FMT
}  // namespace
}  // namespace vx
