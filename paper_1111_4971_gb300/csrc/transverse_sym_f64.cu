// FP64 instantiation of the pipe-operator transverse stage.
#define PP_TS_TYPE double
#include "transverse_sym.cu"
