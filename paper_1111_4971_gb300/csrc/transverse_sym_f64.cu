// FP64 instantiation of the pipe-operator transverse stage.
#define PP_TS_TYPE double
#define PP_TS_F64_UNIT
#include "transverse_sym.cu"
