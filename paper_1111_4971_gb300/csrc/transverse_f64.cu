// FP64 instantiation of the transverse stage.
#define PP_T_TYPE double
#include "transverse.cu"
