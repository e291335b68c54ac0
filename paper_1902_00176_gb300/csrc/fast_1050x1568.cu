// fast_1050x1568.cu -- register-resident passes for the 1050 x 1568 padded domain
// (row schedule RowShape<1568, 56, 28, 4>, column schedule ColShape<1050, 30, 35, 6>).
#include "fast_kernels.cuh"

namespace gfc {

using RowS_1050x1568 = RowShape<1568, 56, 28, 4>;
using ColS_1050x1568 = ColShape<1050, 30, 35, 6>;

cudaError_t fast_run_1050x1568(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1, void* out0,
                          void* out1, int nf, cudaStream_t st, const EditArgs* ed) {
  return run_fast_shape<RowS_1050x1568, ColS_1050x1568>(P, bf, mode, in0, in1, out0, out1, nf, st, ed);
}

size_t fast_zbuf_1050x1568(int H) { return fast_zbuf_elems_for<RowS_1050x1568>(H); }

int fast_items_1050x1568() { return RowS_1050x1568::F; }

}  // namespace gfc
