// formats_small.cu -- compile-time-composed kernels for the 64^3 and 512^3
// formats (the paper's Sec. 4 metaprogramming system generates one
// intersection function per level; here C++ templates compose them).
#include "trace.cuh"

namespace vx {
namespace {
#define VX_FMT(id, text, ...)                                                     \
    const KernelSet ks_##id = make_kernel_set<Format<__VA_ARGS__>>(text);        \
    KernelSetRegistrar reg_##id(&ks_##id);

VX_FMT(s4r2, "S(4) R(2,2,2)", Svo<4>, Raw<2, 2, 2>)
VX_FMT(s3r3, "S(3) R(3,3,3)", Svo<3>, Raw<3, 3, 3>)
VX_FMT(r4s2g3, "R(4,4,4) S(2) G(3)", Raw<4, 4, 4>, Svo<2>, Dag<3>)
VX_FMT(r3r3r3, "R(3,3,3) R(3,3,3) R(3,3,3)", Raw<3, 3, 3>, Raw<3, 3, 3>, Raw<3, 3, 3>)
VX_FMT(r4g5, "R(4,4,4) G(5)", Raw<4, 4, 4>, Dag<5>)
VX_FMT(r2g7, "R(2,2,2) G(7)", Raw<2, 2, 2>, Dag<7>)
VX_FMT(r4s5, "R(4,4,4) S(5)", Raw<4, 4, 4>, Svo<5>)
#undef VX_FMT
}  // namespace
}  // namespace vx
