// One instantiation of the persistent refinement kernel (A_u stored as
// double, factors stored as __half); split per file so the instantiations
// compile in parallel.
#include "refine_impl.cuh"

namespace msir {
template <> void* refine_entry<double, __half>() { return (void*)refine_kernel<double, __half>; }
}  // namespace msir
