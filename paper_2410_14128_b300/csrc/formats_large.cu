// formats_large.cu -- compile-time-composed kernels for the 2048^3 format
// sweep: the Table 2 formats whose Raw levels branch 2^1..2^4 per axis, plus
// one format with 2^2 and 2^1 Raw levels.
#include "trace.cuh"

namespace vx {
namespace {
#define VX_FMT(id, text, ...)                                                     \
    const KernelSet ks_##id = make_kernel_set<Format<__VA_ARGS__>>(text);        \
    KernelSetRegistrar reg_##id(&ks_##id);

VX_FMT(r4r3g4, "R(4,4,4) R(3,3,3) G(4)", Raw<4, 4, 4>, Raw<3, 3, 3>, Dag<4>)
VX_FMT(r4s3g4, "R(4,4,4) S(3) G(4)", Raw<4, 4, 4>, Svo<3>, Dag<4>)
VX_FMT(r4r4r3, "R(4,4,4) R(4,4,4) R(3,3,3)", Raw<4, 4, 4>, Raw<4, 4, 4>, Raw<3, 3, 3>)
VX_FMT(r4s7, "R(4,4,4) S(7)", Raw<4, 4, 4>, Svo<7>)
VX_FMT(r4g7, "R(4,4,4) G(7)", Raw<4, 4, 4>, Dag<7>)
VX_FMT(r3g8, "R(3,3,3) G(8)", Raw<3, 3, 3>, Dag<8>)
VX_FMT(s7g4, "S(7) G(4)", Svo<7>, Dag<4>)
VX_FMT(s5g6, "S(5) G(6)", Svo<5>, Dag<6>)
VX_FMT(s3g8, "S(3) G(8)", Svo<3>, Dag<8>)
VX_FMT(s11, "S(11)", Svo<11>)
VX_FMT(g11, "G(11)", Dag<11>)
VX_FMT(r2r1s4g4, "R(2,2,2) R(1,1,1) S(4) G(4)", Raw<2, 2, 2>, Raw<1, 1, 1>, Svo<4>, Dag<4>)
#undef VX_FMT
}  // namespace
}  // namespace vx
