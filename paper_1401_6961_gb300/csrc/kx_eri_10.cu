// kx_eri_10.cu -- McMurchie-Davidson class kernels with bra pair class
// (la, lb) = (1, 0): the nine ket classes (lc, ld), FP64 and FP32.  One
// translation unit per bra class so that the 81 classes compile in parallel.
#include "kx_eri_impl.cuh"

namespace kx {
KX_ERI_DISPATCH(1, 0)
}  // namespace kx
