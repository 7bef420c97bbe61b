// Kernel instantiations for one lattice pair (one translation unit per pair
// so that the library compiles in parallel).
#include "aux_kernels.cuh"

namespace lbpf {
const Launchers* launchers_d2q9(int precision) { return launchers_for<LBPF_D2Q9_D2Q5>(precision); }
}  // namespace lbpf
