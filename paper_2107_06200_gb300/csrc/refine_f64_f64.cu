// One instantiation of the persistent refinement kernel (A_u stored as
// double, factors stored as double); split per file so the instantiations
// compile in parallel.
#include "refine_impl.cuh"

namespace msir {
template <> void* refine_entry<double, double>() { return (void*)refine_kernel<double, double>; }
}  // namespace msir
