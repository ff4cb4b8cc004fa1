// One instantiation of the persistent refinement kernel (A_u stored as
// float, factors stored as double); split per file so the instantiations
// compile in parallel.
#include "refine_impl.cuh"

namespace msir {
template <> void* refine_entry<float, double>() { return (void*)refine_kernel<float, double>; }
}  // namespace msir
