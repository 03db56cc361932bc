// FP64 instantiation of the z-axis transforms.
#define PP_Z_TYPE double
#define PP_Z_F64_UNIT
#include "zfft.cu"
