// Kernel instantiations for one lattice pair (one translation unit per pair
// so that the library compiles in parallel).
#include "aux_kernels.cuh"

namespace lbpf {
const Launchers* launchers_d3q27(int precision) { return launchers_for<LBPF_D3Q27_D3Q7>(precision); }
}  // namespace lbpf
