// pa_batch_hi.cu -- part 1 of the batched sweep kernel (pa_batch.cuh): the
// runs with five to seven bits per state (q = 17..128), compiled apart from
// part 0 so that each part keeps its own register allocation and the two
// translation units build in parallel.
#include "pa_batch.cuh"

namespace pa {

BatchSweepFn batch_sweep_kernel_hi() { return k_batch_sweep<1>; }

}  // namespace pa
