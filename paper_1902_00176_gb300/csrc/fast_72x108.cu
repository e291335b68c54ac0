// fast_72x108.cu -- register-resident passes for the 72 x 108 padded domain
// (row schedule RowShape<108, 9, 12, 10>, column schedule ColShape<72, 8, 9, 16>).
#include "fast_kernels.cuh"

namespace gfc {

using RowS_72x108 = RowShape<108, 9, 12, 10>;
using ColS_72x108 = ColShape<72, 8, 9, 16>;

cudaError_t fast_run_72x108(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1, void* out0,
                          void* out1, int nf, cudaStream_t st, const EditArgs* ed) {
  return run_fast_shape<RowS_72x108, ColS_72x108>(P, bf, mode, in0, in1, out0, out1, nf, st, ed);
}

size_t fast_zbuf_72x108(int H) { return fast_zbuf_elems_for<RowS_72x108>(H); }

int fast_items_72x108() { return RowS_72x108::F; }

}  // namespace gfc
