// Kernel instantiations for one lattice pair and one storage precision,
// chosen at compile time by LBPF_LAT (an lbpf_lattice) and LBPF_PREC (an
// lbpf_precision).  The library is built from one object of this file per
// pair and precision, compiled in parallel; lbpf_launchers.cu dispatches.
#include "aux_kernels.cuh"

#if !defined(LBPF_LAT) || !defined(LBPF_PREC)
#error "compile with -DLBPF_LAT=<lattice pair> -DLBPF_PREC=<precision>"
#endif

namespace lbpf {

template <int P> struct StoreOf;
template <> struct StoreOf<LBPF_FP64> { using type = StoreF64; };
template <> struct StoreOf<LBPF_FP32> { using type = StoreF32; };
template <> struct StoreOf<LBPF_FP32_FP16DEV> { using type = StoreF16; };
template <> struct StoreOf<LBPF_FP32_BF16DEV> { using type = StoreB16; };
template <> struct StoreOf<LBPF_FP32_FP16DEV_SR> { using type = StoreF16SR; };

#define LBPF_LAUNCHERS_NAME2(l, p) launchers_l##l##_p##p
#define LBPF_LAUNCHERS_NAME(l, p) LBPF_LAUNCHERS_NAME2(l, p)

const Launchers* LBPF_LAUNCHERS_NAME(LBPF_LAT, LBPF_PREC)()
{
    return LauncherImpl<typename Pair<LBPF_LAT>::P, typename Pair<LBPF_LAT>::U,
                        typename StoreOf<LBPF_PREC>::type>::get();
}

}  // namespace lbpf
