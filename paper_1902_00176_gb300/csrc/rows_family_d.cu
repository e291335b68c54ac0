// rows_family_d.cu -- register-resident row passes for row lengths 784 882 980 1080
// (schedules N = R1 x R2, F transforms per block; recursive column solve only).
#include "rows_family.cuh"

namespace gfc {

GFC_ROW_SHAPE(784,28,28,4)
GFC_ROW_SHAPE(882,21,42,3)
GFC_ROW_SHAPE(980,28,35,3)
GFC_ROW_SHAPE(1080,30,36,3)

}  // namespace gfc
