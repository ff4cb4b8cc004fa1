// One instantiation of the persistent refinement kernel (A_u stored as
// float, factors stored as __half); split per file so the instantiations
// compile in parallel.
#include "refine_impl.cuh"

namespace msir {
template <> void* refine_entry<float, __half>() { return (void*)refine_kernel<float, __half>; }
}  // namespace msir
