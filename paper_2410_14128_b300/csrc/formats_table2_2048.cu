// formats_table2_2048.cu -- compile-time-composed kernels for the 2048^3
// formats of Table 2 outside the sweep of formats_large.cu: the DF formats
// (labels 1, 2, 6-9) and the Raw levels wider than 2^4 (12, 13, 15).
#include "trace.cuh"

namespace vx {
namespace {
#define VX_FMT(id, text, ...)                                                     \
    const KernelSet ks_##id = make_kernel_set<Format<__VA_ARGS__>>(text);        \
    KernelSetRegistrar reg_##id(&ks_##id);

VX_FMT(t01, "D(4,4,4,6) D(3,3,3,6) G(4)", Df<4, 4, 4, 6>, Df<3, 3, 3, 6>, Dag<4>)
VX_FMT(t02, "D(4,4,4,6) R(3,3,3) G(4)", Df<4, 4, 4, 6>, Raw<3, 3, 3>, Dag<4>)
VX_FMT(t06, "D(4,4,4,6) S(7)", Df<4, 4, 4, 6>, Svo<7>)
VX_FMT(t07, "D(4,4,4,6) G(7)", Df<4, 4, 4, 6>, Dag<7>)
VX_FMT(t08, "D(6,6,6,6) S(5)", Df<6, 6, 6, 6>, Svo<5>)
VX_FMT(t09, "D(6,6,6,6) G(5)", Df<6, 6, 6, 6>, Dag<5>)
VX_FMT(t12, "R(6,6,6) S(5)", Raw<6, 6, 6>, Svo<5>)
VX_FMT(t13, "R(6,6,6) G(5)", Raw<6, 6, 6>, Dag<5>)
VX_FMT(t15, "R(8,8,8) G(3)", Raw<8, 8, 8>, Dag<3>)
#undef VX_FMT
}  // namespace
}  // namespace vx
