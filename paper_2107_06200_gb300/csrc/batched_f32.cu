// Batched engine, working precision u0 = fp32.
#include "batched_impl.cuh"

namespace msir {
void* batched_solve_entry_f32() { return (void*)batched_solve_kernel<float>; }
}  // namespace msir
