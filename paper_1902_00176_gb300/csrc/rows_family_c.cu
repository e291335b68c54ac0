// rows_family_c.cu -- register-resident row passes for row lengths 448 500 560 630 700
// (schedules N = R1 x R2, F transforms per block; recursive column solve only).
#include "rows_family.cuh"

namespace gfc {

GFC_ROW_SHAPE(448,16,28,4)
GFC_ROW_SHAPE(500,20,25,5)
GFC_ROW_SHAPE(560,20,28,4)
GFC_ROW_SHAPE(630,21,30,4)
GFC_ROW_SHAPE(700,25,28,4)

}  // namespace gfc
