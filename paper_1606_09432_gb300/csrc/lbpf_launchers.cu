// Dispatch from (lattice pair, precision) to the launchers of the object
// built from lbpf_lattice.cu for that pair and precision.
#include "lbpf_internal.cuh"

namespace lbpf {

#define LBPF_DECL_PAIR(l)                    \
    const Launchers* launchers_l##l##_p0(); \
    const Launchers* launchers_l##l##_p1(); \
    const Launchers* launchers_l##l##_p2(); \
    const Launchers* launchers_l##l##_p3(); \
    const Launchers* launchers_l##l##_p4();
LBPF_DECL_PAIR(0)
LBPF_DECL_PAIR(1)
LBPF_DECL_PAIR(2)
LBPF_DECL_PAIR(3)

const Launchers* launchers_for_pair(int lattice, int precision)
{
    using Fn = const Launchers* (*)();
    static const Fn table[4][5] = {
        {launchers_l0_p0, launchers_l0_p1, launchers_l0_p2, launchers_l0_p3, launchers_l0_p4},
        {launchers_l1_p0, launchers_l1_p1, launchers_l1_p2, launchers_l1_p3, launchers_l1_p4},
        {launchers_l2_p0, launchers_l2_p1, launchers_l2_p2, launchers_l2_p3, launchers_l2_p4},
        {launchers_l3_p0, launchers_l3_p1, launchers_l3_p2, launchers_l3_p3, launchers_l3_p4},
    };
    if (lattice < 0 || lattice > 3 || precision < 0 || precision > 4) return nullptr;
    return table[lattice][precision]();
}

}  // namespace lbpf
