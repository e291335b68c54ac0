// rows_family_f.cu -- register-resident row passes for row lengths 1536 1750 1960 2058
// (schedules N = R1 x R2, F transforms per block; recursive column solve only).
#include "rows_family.cuh"

namespace gfc {

GFC_ROW_SHAPE(1536,32,48,3)
GFC_ROW_SHAPE(1750,35,50,3)
GFC_ROW_SHAPE(1960,35,56,2)
GFC_ROW_SHAPE(2058,42,49,2)

}  // namespace gfc
