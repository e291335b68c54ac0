// rows_family_b.cu -- register-resident row passes for row lengths 252 294 320 360 400
// (schedules N = R1 x R2, F transforms per block; recursive column solve only).
#include "rows_family.cuh"

namespace gfc {

GFC_ROW_SHAPE(252,14,18,7)
GFC_ROW_SHAPE(294,14,21,6)
GFC_ROW_SHAPE(320,16,20,6)
GFC_ROW_SHAPE(360,18,20,6)
GFC_ROW_SHAPE(400,20,20,6)

}  // namespace gfc
