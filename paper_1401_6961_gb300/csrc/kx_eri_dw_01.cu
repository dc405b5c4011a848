// kx_eri_dw_01.cu -- double-word FP32 class kernels (kx_dw.cuh) with bra
// pair class (la, lb) = (0, 1): the ket classes with la+lb+lc+ld <=
// DW_LMAX.  One translation unit per bra class so that they compile in
// parallel.
#include "kx_eri_impl.cuh"

namespace kx {
KX_ERI_DISPATCH_DW(0, 1)
}  // namespace kx
