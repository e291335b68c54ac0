// rows_family_a.cu -- register-resident row passes for row lengths 140 160 180 200 224
// (schedules N = R1 x R2, F transforms per block; recursive column solve only).
#include "rows_family.cuh"

namespace gfc {

GFC_ROW_SHAPE(140,10,14,9)
GFC_ROW_SHAPE(160,10,16,8)
GFC_ROW_SHAPE(180,12,15,8)
GFC_ROW_SHAPE(200,10,20,6)
GFC_ROW_SHAPE(224,14,16,8)

}  // namespace gfc
