// rows_family_e.cu -- register-resident row passes for row lengths 1120 1200 1372 1400
// (schedules N = R1 x R2, F transforms per block; recursive column solve only).
#include "rows_family.cuh"

namespace gfc {

GFC_ROW_SHAPE(1120,28,40,3)
GFC_ROW_SHAPE(1200,30,40,3)
GFC_ROW_SHAPE(1372,28,49,4)
GFC_ROW_SHAPE(1400,35,40,4)

}  // namespace gfc
