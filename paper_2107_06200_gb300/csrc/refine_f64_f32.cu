// One instantiation of the persistent refinement kernel (A_u stored as
// double, factors stored as float); split per file so the instantiations
// compile in parallel.
#include "refine_impl.cuh"

namespace msir {
template <> void* refine_entry<double, float>() { return (void*)refine_kernel<double, float>; }
}  // namespace msir
