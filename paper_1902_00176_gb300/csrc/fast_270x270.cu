// fast_270x270.cu -- register-resident passes for the 270 x 270 padded domain
// (row schedule RowShape<270, 15, 18, 7>, column schedule ColShape<270, 15, 18, 8>).
#include "fast_kernels.cuh"

namespace gfc {

using RowS_270x270 = RowShape<270, 15, 18, 7>;
using ColS_270x270 = ColShape<270, 15, 18, 8>;

cudaError_t fast_run_270x270(gfc_plan* P, const Bufs& bf, int mode, const void* in0, const void* in1, void* out0,
                          void* out1, int nf, cudaStream_t st, const EditArgs* ed) {
  return run_fast_shape<RowS_270x270, ColS_270x270>(P, bf, mode, in0, in1, out0, out1, nf, st, ed);
}

size_t fast_zbuf_270x270(int H) { return fast_zbuf_elems_for<RowS_270x270>(H); }

int fast_items_270x270() { return RowS_270x270::F; }

}  // namespace gfc
