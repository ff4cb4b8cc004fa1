// Batched engine, working precision u0 = fp64.
#include "batched_impl.cuh"

namespace msir {
void* batched_solve_entry_f64() { return (void*)batched_solve_kernel<double>; }
}  // namespace msir
