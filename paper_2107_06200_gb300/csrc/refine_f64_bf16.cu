// One instantiation of the persistent refinement kernel (A_u stored as
// double, factors stored as __nv_bfloat16); split per file so the instantiations
// compile in parallel.
#include "refine_impl.cuh"

namespace msir {
template <> void* refine_entry<double, __nv_bfloat16>() { return (void*)refine_kernel<double, __nv_bfloat16>; }
}  // namespace msir
